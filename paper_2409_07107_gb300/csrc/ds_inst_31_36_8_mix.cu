// Kernel instantiation for 31 bodies, 36 dofs, 8 contact slots, mixed precision.
#include "ds_launch.cuh"

void ds_launch_31_36_8_mix(const KArgs& a, cudaStream_t s) { ds::launch_env<31, 36, 8, float>(a, s); }
void ds_pipeline_31_36_8_mix(const KArgs& a, cudaStream_t s) { ds::launch_pipeline<31, 36, 8, float>(a, s); }
void ds_tape_31_36_8_mix(const KArgs& a, cudaStream_t s) { ds::launch_tape<31, 36, 8, float>(a, s); }
unsigned ds_check_31_36_8_mix() { return ds::check_read(); }
