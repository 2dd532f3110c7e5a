// Kernel instantiation for 1 bodies, 6 dofs, 1 contact slots, FP64.
#include "ds_launch.cuh"

void ds_launch_1_6_1_f64(const KArgs& a, cudaStream_t s) { ds::launch_env<1, 6, 1, double>(a, s); }
void ds_pipeline_1_6_1_f64(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<1, 6, 1, double>(a, s); }
void ds_tape_1_6_1_f64(const KArgs& a, cudaStream_t s) { ds::launch_tape<1, 6, 1, double>(a, s); }
unsigned ds_check_1_6_1_f64() { return ds::check_read(); }
