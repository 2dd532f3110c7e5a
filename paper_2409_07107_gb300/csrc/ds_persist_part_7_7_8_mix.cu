// Steps of the persistent kernel's per-env path for the 7-dof arm with 8 contact slots, mixed
// precision (relocatable device code; see ds_persist.cuh).
#define DS_PERSIST_PART
#include "ds_persist.cuh"

namespace ds {
DS_PERSIST_FORWARD(7, 7, 8, float)
DS_PERSIST_SOLVE(7, 7, 8, float)
DS_PERSIST_FINISH(7, 7, 8, float)
}  // namespace ds

unsigned ds_check_persist_7_7_8_mix() { return ds::check_read(); }
