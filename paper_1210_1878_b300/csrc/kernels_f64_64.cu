// Kernel instantiations (one translation unit per precision and strip width,
// compiled in parallel).
#include "kernel_table.cuh"

namespace pcg {

KernelSet kernels_f64_64(int pattern, int q) { return pick_tx<double, 64>(pattern, q); }

}  // namespace pcg
