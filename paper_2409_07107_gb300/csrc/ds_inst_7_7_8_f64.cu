// Kernel instantiation for 7 bodies, 7 dofs, 8 contact slots, FP64.
#include "ds_launch.cuh"

void ds_launch_7_7_8_f64(const KArgs& a, cudaStream_t s) { ds::launch_env<7, 7, 8, double>(a, s); }
void ds_pipeline_7_7_8_f64(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<7, 7, 8, double>(a, s); }
void ds_tape_7_7_8_f64(const KArgs& a, cudaStream_t s) { ds::launch_tape<7, 7, 8, double>(a, s); }
unsigned ds_check_7_7_8_f64() { return ds::check_read(); }
