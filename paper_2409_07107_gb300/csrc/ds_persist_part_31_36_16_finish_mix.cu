// Steps of the persistent kernel's per-env path for the 36-dof humanoid (31 bodies, 16 slots), its finish, mixed
// precision (relocatable device code; see ds_persist.cuh).
#define DS_PERSIST_PART
#include "ds_persist.cuh"

namespace ds {
DS_PERSIST_FINISH(31, 36, 16, float)
}  // namespace ds

unsigned ds_check_persist_31_36_16_finish_mix() { return ds::check_read(); }
