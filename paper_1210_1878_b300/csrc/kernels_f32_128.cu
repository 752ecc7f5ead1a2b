// Kernel instantiations (one translation unit per precision and strip width,
// compiled in parallel).
#include "kernel_table.cuh"

namespace pcg {

KernelSet kernels_f32_128(int pattern, int q) { return pick_tx<float, 128>(pattern, q); }

}  // namespace pcg
