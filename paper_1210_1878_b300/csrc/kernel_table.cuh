// Kernel sets: the instantiations of the two loop kernels (per launch kind)
// and of the small kernels for one precision, strip width and pattern of Z.
// Included by the kernels_*.cu translation units only.
#pragma once

#include "handle.cuh"

namespace pcg {

template <typename T, int TX, class P>
KernelSet make_set() {
  KernelSet k;
  k.k1[K1_ITER] = (const void *)k_stencil<T, TX, K1_ITER, false>;
  k.k1[K1_RESID_INIT] = (const void *)k_stencil<T, TX, K1_RESID_INIT, false>;
  k.k1[K1_RESID_CHECK] = (const void *)k_stencil<T, TX, K1_RESID_CHECK, false>;
  k.k1[K1_SPMV] = (const void *)k_stencil<T, TX, K1_SPMV, false>;
  k.k2[K2_ITER] = (const void *)k_precond<T, TX, P, K2_ITER, false>;
  k.k2[K2_INIT] = (const void *)k_precond<T, TX, P, K2_INIT, false>;
  k.k2[K2_APPLY] = (const void *)k_precond<T, TX, P, K2_APPLY, false>;
  if constexpr (sizeof(T) == 4) {   // batches' binary32 inner iterations claim units
    k.k1_claim = (const void *)k_stencil<T, TX, K1_ITER, true>;
    k.k2_claim = (const void *)k_precond<T, TX, P, K2_ITER, true>;
  }
  k.fin = (const void *)k_finalize<T, TX>;
  k.pack = (const void *)k_pack<T, double, TX>;
  k.unpack = (const void *)k_unpack<T, double>;
  k.smem1 = K1Geom<T, TX>::SMEM;
  k.smem2 = K2Geom<T, TX, P>::SMEM;
  k.tx = TX;
  k.tb = K1Geom<T, TX>::NT;
  k.rb1 = K1Geom<T, TX>::RB;
  k.rb2 = K2Geom<T, TX, P>::RB;
  k.ws = K1Geom<T, TX>::WS; k.we = K1Geom<T, TX>::WE; k.wt = K1Geom<T, TX>::WT;
  k.wr = K2Geom<T, TX, P>::WR; k.wz = K2Geom<T, TX, P>::WZ;
  static_assert(K1Geom<T, TX>::NT == K2Geom<T, TX, P>::NT, "both kernels use one block size");
  k.ok = true;
  return k;
}

template <typename T, int TX>
KernelSet pick_tx(int pattern, int q) {
  switch (pattern) {
    case PCG_PAT_DIAG: return make_set<T, TX, Pat<PCG_PAT_DIAG, 0>>();
    case PCG_PAT_TRIL_A: return make_set<T, TX, Pat<PCG_PAT_TRIL_A, 0>>();
    case PCG_PAT_TRIL_A2: return make_set<T, TX, Pat<PCG_PAT_TRIL_A2, 0>>();
    case PCG_PAT_BAND_T:
      switch (q) {
        case 1: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 1>>();
        case 2: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 2>>();
        case 3: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 3>>();
        case 4: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 4>>();
        case 5: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 5>>();
        case 6: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 6>>();
        case 7: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 7>>();
        case 8: return make_set<T, TX, Pat<PCG_PAT_BAND_T, 8>>();
        default: break;
      }
      break;
    default: break;
  }
  return KernelSet{};
}

}  // namespace pcg
