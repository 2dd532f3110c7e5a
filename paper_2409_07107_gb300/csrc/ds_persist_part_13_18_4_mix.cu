// Steps of the persistent kernel's per-env path for the 18-dof quadruped (13 bodies, 4 slots), mixed
// precision (relocatable device code; see ds_persist.cuh).
#define DS_PERSIST_PART
#include "ds_persist.cuh"

namespace ds {
DS_PERSIST_FORWARD(13, 18, 4, float)
DS_PERSIST_SOLVE(13, 18, 4, float)
DS_PERSIST_FINISH(13, 18, 4, float)
}  // namespace ds

unsigned ds_check_persist_13_18_4_mix() { return ds::check_read(); }
