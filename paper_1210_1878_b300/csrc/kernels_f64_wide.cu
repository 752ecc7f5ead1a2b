// Kernel instantiations (one translation unit per precision and strip width,
// compiled in parallel).
#include "kernel_table.cuh"

namespace pcg {

KernelSet kernels_f64_wide(int tx, int pattern) {
  if (tx == 124 && pattern == PCG_PAT_TRIL_A) return make_set<double, 124, Pat<PCG_PAT_TRIL_A, 0>>();
  if (tx == 92 && pattern == PCG_PAT_TRIL_A2) return make_set<double, 92, Pat<PCG_PAT_TRIL_A2, 0>>();
  return KernelSet{};
}

}  // namespace pcg
