// Kernel instantiation for 31 bodies, 36 dofs, 16 contact slots, FP64.
#include "ds_launch.cuh"

void ds_launch_31_36_16_f64(const KArgs& a, cudaStream_t s) { ds::launch_env<31, 36, 16, double>(a, s); }
void ds_pipeline_31_36_16_f64(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<31, 36, 16, double>(a, s); }
void ds_tape_31_36_16_f64(const KArgs& a, cudaStream_t s) { ds::launch_tape<31, 36, 16, double>(a, s); }
unsigned ds_check_31_36_16_f64() { return ds::check_read(); }
