// Kernel instantiation for 1 bodies, 6 dofs, 1 contact slots, mixed precision.
#include "ds_launch.cuh"

void ds_launch_1_6_1_mix(const KArgs& a, cudaStream_t s) { ds::launch_env<1, 6, 1, float>(a, s); }
void ds_pipeline_1_6_1_mix(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<1, 6, 1, float>(a, s); }
void ds_tape_1_6_1_mix(const KArgs& a, cudaStream_t s) { ds::launch_tape<1, 6, 1, float>(a, s); }
unsigned ds_check_1_6_1_mix() { return ds::check_read(); }
