// Kernel instantiation for 7 bodies, 7 dofs, 1 contact slots, mixed precision.
#include "ds_launch.cuh"

void ds_launch_7_7_1_mix(const KArgs& a, cudaStream_t s) { ds::launch_env<7, 7, 1, float>(a, s); }
void ds_pipeline_7_7_1_mix(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<7, 7, 1, float>(a, s); }
void ds_tape_7_7_1_mix(const KArgs& a, cudaStream_t s) { ds::launch_tape<7, 7, 1, float>(a, s); }
unsigned ds_check_7_7_1_mix() { return ds::check_read(); }
