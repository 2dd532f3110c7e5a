// Kernel instantiation for 13 bodies, 18 dofs, 4 contact slots, FP64.
#include "ds_launch.cuh"

void ds_launch_13_18_4_f64(const KArgs& a, cudaStream_t s) { ds::launch_env<13, 18, 4, double>(a, s); }
void ds_pipeline_13_18_4_f64(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<13, 18, 4, double>(a, s); }
void ds_tape_13_18_4_f64(const KArgs& a, cudaStream_t s) { ds::launch_tape<13, 18, 4, double>(a, s); }
unsigned ds_check_13_18_4_f64() { return ds::check_read(); }
