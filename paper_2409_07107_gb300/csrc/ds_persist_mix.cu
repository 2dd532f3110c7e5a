// Persistent kernel over the shapes of a batch that mixes a 7-dof arm (8 contact slots), an
// 18-dof quadruped (13 bodies, 4 slots) and a 36-dof humanoid (31 bodies, 16 slots), mixed precision
// (the only precision it is compiled for: each shape's per-env path is one large function, and the
// three of them take minutes to compile).  Relocatable device code: the per-shape steps come from
// the ds_persist_part_* units.
#include "ds_persist.cuh"

unsigned ds_check_persist_7_7_8_mix();
unsigned ds_check_persist_13_18_4_mix();
unsigned ds_check_persist_31_36_16_fwd_mix();
unsigned ds_check_persist_31_36_16_solve_mix();
unsigned ds_check_persist_31_36_16_finish_mix();

namespace {
using Kern = void (*)(const KArgs&, const PArgs&, cudaStream_t);
const Kern kLaunch = ds::launch_persist<float, ds::PShape<7, 7, 8>, ds::PShape<13, 18, 4>, ds::PShape<31, 36, 16>>;
unsigned check() {
  return ds::check_read() + ds_check_persist_7_7_8_mix() + ds_check_persist_13_18_4_mix() +
         ds_check_persist_31_36_16_fwd_mix() + ds_check_persist_31_36_16_solve_mix() +
         ds_check_persist_31_36_16_finish_mix();
}
}  // namespace

const ds_persist_entry* ds_persist_mix() {
  static const ds_persist_entry e =
      ds::persist_entry<float, ds::PShape<7, 7, 8>, ds::PShape<13, 18, 4>, ds::PShape<31, 36, 16>>(DS_MIXED, kLaunch, check);
  return &e;
}
