// Table of compiled (bodies, dofs, contact slots, precision) shapes.
#include "ds_common.cuh"

#define DS_DECL(NB, NV, NS)                                                \
  void ds_launch_##NB##_##NV##_##NS##_f64(const KArgs&, cudaStream_t);       \
  void ds_launch_##NB##_##NV##_##NS##_mix(const KArgs&, cudaStream_t);       \
  void ds_pipeline_##NB##_##NV##_##NS##_f64(const KArgs&, cudaStream_t);     \
  void ds_pipeline_##NB##_##NV##_##NS##_mix(const KArgs&, cudaStream_t);   \
  void ds_tape_##NB##_##NV##_##NS##_f64(const KArgs&, cudaStream_t);         \
  void ds_tape_##NB##_##NV##_##NS##_mix(const KArgs&, cudaStream_t);         \
  unsigned ds_check_##NB##_##NV##_##NS##_f64();                              \
  unsigned ds_check_##NB##_##NV##_##NS##_mix();
#define DS_ROW(NB, NV, NS)                                                                          \
  {NB, NV, NS, DS_FP64, ds_launch_##NB##_##NV##_##NS##_f64, ds_pipeline_##NB##_##NV##_##NS##_f64,     \
   ds_tape_##NB##_##NV##_##NS##_f64, ds_check_##NB##_##NV##_##NS##_f64},                              \
  {NB, NV, NS, DS_MIXED, ds_launch_##NB##_##NV##_##NS##_mix, ds_pipeline_##NB##_##NV##_##NS##_mix,    \
   ds_tape_##NB##_##NV##_##NS##_mix, ds_check_##NB##_##NV##_##NS##_mix},

#include "ds_shapes.inc"

static const ds_kernel_entry kTable[] = {
#define DS_SHAPE(NB, NV, NS) DS_ROW(NB, NV, NS)
#include "ds_shapes_list.inc"
#undef DS_SHAPE
};

const ds_kernel_entry* ds_find_kernel(int nb, int nv, int ns, int precision) {
  for (const ds_kernel_entry& k : kTable)
    if (k.nb == nb && k.nv == nv && k.ns == ns && k.precision == precision) return &k;
  return nullptr;
}

// The compiled shape for a model whose envs use the leading `slots` contact slots of a batch with
// ncmax slots: the fewest slots S with slots <= S <= ncmax (the kernel reads slots 0 .. S-1 only).
const ds_kernel_entry* ds_fit_kernel(int nb, int nv, int slots, int ncmax, int precision) {
  const ds_kernel_entry* best = nullptr;
  for (const ds_kernel_entry& k : kTable)
    if (k.nb == nb && k.nv == nv && k.precision == precision && k.ns >= slots && k.ns <= ncmax &&
        (!best || k.ns < best->ns))
      best = &k;
  return best;
}

const ds_persist_entry* ds_persist_mix();

// The persistent kernel is compiled for the mixed-precision form only.
const ds_persist_entry* ds_persist_kernel(int precision) {
  return precision == DS_MIXED ? ds_persist_mix() : nullptr;
}

unsigned long long ds_check_sum() {
  unsigned long long n = 0;
  for (const ds_kernel_entry& k : kTable) n += k.check();
  n += ds_persist_mix()->check();
  return n;
}
