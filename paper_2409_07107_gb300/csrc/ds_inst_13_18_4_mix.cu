// Kernel instantiation for 13 bodies, 18 dofs, 4 contact slots, mixed precision.
#include "ds_launch.cuh"

void ds_launch_13_18_4_mix(const KArgs& a, cudaStream_t s) { ds::launch_env<13, 18, 4, float>(a, s); }
void ds_pipeline_13_18_4_mix(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<13, 18, 4, float>(a, s); }
void ds_tape_13_18_4_mix(const KArgs& a, cudaStream_t s) { ds::launch_tape<13, 18, 4, float>(a, s); }
unsigned ds_check_13_18_4_mix() { return ds::check_read(); }
