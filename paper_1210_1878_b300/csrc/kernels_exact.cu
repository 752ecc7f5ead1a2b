// Kernel instantiations (one translation unit per precision and strip width,
// compiled in parallel).
#include "kernel_table.cuh"

namespace pcg {

KernelSet kernels_f64_exact(int tx, int pattern) {
  if (tx == 60 && pattern == PCG_PAT_TRIL_A2) return make_set<double, 60, Pat<PCG_PAT_TRIL_A2, 0>>();
  if (tx == 62 && pattern == PCG_PAT_TRIL_A) return make_set<double, 62, Pat<PCG_PAT_TRIL_A, 0>>();
  return KernelSet{};
}

KernelSet kernels_f32_exact(int tx, int pattern) {
  if (tx == 124 && pattern == PCG_PAT_TRIL_A2) return make_set<float, 124, Pat<PCG_PAT_TRIL_A2, 0>>();
  if (tx == 124 && pattern == PCG_PAT_TRIL_A) return make_set<float, 124, Pat<PCG_PAT_TRIL_A, 0>>();
  return KernelSet{};
}

}  // namespace pcg
