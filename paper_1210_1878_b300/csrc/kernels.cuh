// Kernel bodies of libpcg. See device.cuh for the data layout and the
// execution scheme. Everything here is templated on the storage/compute type
// T (double for the binary64 solve, float for the inner solves of the mixed
// precision mode) and on the strip width TX (= threads per CTA).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pcg.h"
#include "device.cuh"

namespace pcg {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Bulk asynchronous copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned) from global memory into this CTA's shared memory; completion is
// counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for a phase of an mbarrier, giving up after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > timeout_ns) return false;
  }
}

// ------------------------------------------------------------ patterns of Z
// Slot planes (offset of the row m of column k's entry, relative to k) and
// side-table entries for the periodic east neighbours of the last columns.
// The plane order matches slot_set() of the host build.
template <int PAT, int Q>
struct Pat;
template <>
struct Pat<PCG_PAT_DIAG, 0> {
  static constexpr int NZ = 0, NW = 0, LD = 0, R = 0;
  __device__ static constexpr int dx(int) { return 0; }
  __device__ static constexpr int dy(int) { return 0; }
  __device__ static constexpr int wcol(int) { return 0; }
  __device__ static constexpr int wdx(int) { return 0; }
};
template <>
struct Pat<PCG_PAT_TRIL_A, 0> {
  static constexpr int NZ = 2, NW = 1, LD = 1, R = 1;
  __device__ static constexpr int dx(int s) { return s == 0 ? -1 : 0; }
  __device__ static constexpr int dy(int s) { return s == 0 ? 0 : -1; }
  __device__ static constexpr int wcol(int) { return 0; }
  __device__ static constexpr int wdx(int) { return 1; }
};
template <>
struct Pat<PCG_PAT_TRIL_A2, 0> {
  static constexpr int NZ = 6, NW = 3, LD = 2, R = 2;
  __device__ static constexpr int dx(int s) {
    return s == 0 ? -2 : s == 1 ? -1 : s == 2 ? -1 : s == 3 ? 0 : s == 4 ? 1 : 0;
  }
  __device__ static constexpr int dy(int s) { return s <= 1 ? 0 : s <= 4 ? -1 : -2; }
  __device__ static constexpr int wcol(int w) { return w == 2 ? 1 : 0; }
  __device__ static constexpr int wdx(int w) { return w == 0 ? 1 : 2; }
};
template <int Q>
struct Pat<PCG_PAT_BAND_T, Q> {
  static constexpr int NZ = Q, NW = 0, LD = 0, R = Q;
  __device__ static constexpr int dx(int s) { return -(s + 1); }
  __device__ static constexpr int dy(int) { return 0; }
  __device__ static constexpr int wcol(int) { return 0; }
  __device__ static constexpr int wdx(int) { return 0; }
};

__host__ __device__ constexpr int round_up_c(int v, int a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------ stores
// Store one value of column `col` (0 <= col < nx) of a row, together with its
// periodic copies in the ghost columns.
template <typename T>
__device__ __forceinline__ void store_dup(T *row, int col, int nx, T v) {
  row[col] = v;
  if (col < GHOST)
    for (int c = col + nx; c < nx + GHOST; c += nx) row[c] = v;
  if (col >= nx - GHOST)
    for (int c = col - nx; c >= -GHOST; c -= nx) row[c] = v;
}

// ------------------------------------------------------------ reductions
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int i = 0; i < NW; ++i) { sa += red[2 * i]; sb += red[2 * i + 1]; }
    a = sa; b = sb;
  }
}

// Write this unit's partials; return true (in every thread) if this CTA is the
// last of its grid to arrive, in which case (sa, sb) hold the grid's totals in
// thread 0, summed in unit order.
template <int NT>
__device__ __forceinline__ bool grid_reduce2(double &sa, double &sb, double *partial, int u, int n_units,
                                             uint32_t *counter, double *red, int *flag) {
  block_sum2<NT>(sa, sb, red);
  if (threadIdx.x == 0) {
    partial[2 * u] = sa;
    partial[2 * u + 1] = sb;
    __threadfence();
    const uint32_t prev = atomicAdd(counter, 1u);
    *flag = (prev == (uint32_t)(n_units - 1));
  }
  __syncthreads();
  if (!*flag) return false;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < n_units; t += NT) {
    a += __ldcg(partial + 2 * t);
    b += __ldcg(partial + 2 * t + 1);
  }
  block_sum2<NT>(a, b, red);
  if (threadIdx.x == 0) {
    sa = a; sb = b;
    atomicExch(counter, 0u);
  }
  return true;
}

__device__ __forceinline__ void grid_finished(SolveState *st, LaunchState *ls, int status, bool may_set_cond,
                                             const KParams &p) {
  if (status != PCG_OK) atomicCAS(&st->status, PCG_OK, status);
  st->done = 1;
  __threadfence();
  const int prev = atomicSub(&ls->active, 1);
  if (prev == 1 && may_set_cond && p.use_cond) cudaGraphSetConditional(ls->cond, 0);
}

__device__ __forceinline__ void flag_timeout(SolveState *st) { atomicCAS(&st->status, PCG_OK, PCG_ETIMEOUT); }

// ------------------------------------------------------------ kernel 1
// Stencil pass (Section 3, Eq. 9 in SPD form). Kinds:
//  K1_ITER        d' = s + beta d; x += pending d; q = A d'; sum d'.q
//  K1_RESID_INIT  r = b - A x; sums r.r and b.b
//  K1_RESID_CHECK r = b - A x; sum r.r (true residual)
//  K1_SPMV        q = A v (v in d[0])
template <typename T, int TX>
struct K1Geom {
  static constexpr int AL = 16 / (int)sizeof(T);     // elements per 16 bytes
  static constexpr int H = AL;                       // halo of the centre fields (>= 1)
  static constexpr int WS = TX + 2 * H;              // s, d_old / x / v: [i0-H, i0+TX+H)
  static constexpr int WE = TX + H;                  // c_e: [i0-H, i0+TX)
  static constexpr int WT = TX;                      // c_n, a, x / b
  static constexpr int NST = 6;                      // ring slots (3 live rows + 3 ahead)
  static constexpr int OFF_S = 0, OFF_D = WS, OFF_E = 2 * WS, OFF_N = 2 * WS + WE, OFF_A = OFF_N + WT,
                       OFF_X = OFF_A + WT, SLOT = OFF_X + WT;
  static constexpr int WDN = TX + 2;                 // d' ring: [i0-1, i0+TX+1)
  static constexpr size_t SMEM = 128 + sizeof(T) * ((size_t)NST * SLOT + 3 * WDN) + 16 * 2 * (TX / 32) + 64;
};

template <typename T, int TX>
__global__ void __launch_bounds__(TX) k_stencil(KParams p) {
  using G = K1Geom<T, TX>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  T *ring = reinterpret_cast<T *>(smem_raw + 128);
  T *dn = ring + (size_t)G::NST * G::SLOT;
  double *red = reinterpret_cast<double *>(dn + 3 * G::WDN);
  int *flag = reinterpret_cast<int *>(red + 2 * (TX / 32));

  const Unit un = p.units[blockIdx.x];
  const GridDev<T> &gd = reinterpret_cast<const GridDev<T> *>(p.grids)[un.g];
  SolveState *st = gd.st;
  LaunchState *ls = p.ls;
  const int kind = p.kind;

  if (p.guard && blockIdx.x == 0 && threadIdx.x == 0) {
    // loop exit and runaway guard (count and wall clock) of the loop graph
    const int l = atomicAdd(&ls->launches, 1) + 1;
    const uint64_t now = global_ns();
    if (ls->t0_ns == 0) ls->t0_ns = now;
    const bool late = now - ls->t0_ns > ls->budget_ns;
    if (late) ls->timed_out = 1;
    if (l > ls->max_launches || late || atomicAdd(&ls->active, 0) == 0) {
      ls->stop = 1;
      if (p.use_cond) cudaGraphSetConditional(ls->cond, 0);
    }
  }
  if ((kind == K1_ITER || kind == K1_RESID_INIT) && *(volatile int32_t *)&st->done) return;
  if (kind == K1_RESID_CHECK && *(volatile int32_t *)&st->retired) return;

  const int nx = gd.nx, ny = gd.ny, pitch = gd.pitch;
  const int i0 = un.sx * TX, j0 = un.sy * gd.ty;
  const int rend = min(j0 + gd.ty, ny);
  const int mlo = j0 - 1, mhi = rend;          // rows streamed: south halo row .. north look-ahead row
  const int tid = threadIdx.x;
  const T beta = (kind == K1_ITER) ? (T)st->beta : (T)0;
  const T pend = (kind == K1_ITER) ? (T)st->pending : (T)0;
  const int dsel = st->dsel;
  const int rsel1 = st->rsel;

  const T *src = (kind == K1_ITER) ? gd.s : (kind == K1_SPMV) ? gd.d[0] : gd.x;
  const T *dold = gd.d[dsel];
  const T *xb = (kind == K1_ITER) ? gd.x : gd.b;

  const bool skip_first = (p.dbg_skip_unit == (int)blockIdx.x);

  auto issue = [&](int m) {
    const int slot = (m - mlo) % G::NST;
    T *sl = ring + (size_t)slot * G::SLOT;
    const size_t rowoff = (size_t)m * pitch;
    uint32_t bytes = G::WS * sizeof(T);
    const bool need_d = (kind == K1_ITER);
    const bool need_n = (m < mhi);
    const bool need_row = (m >= j0 && m < mhi);
    const bool need_x = need_row && kind != K1_SPMV;
    if (need_d) bytes += G::WS * sizeof(T);
    if (need_n) bytes += G::WT * sizeof(T);
    if (need_row) bytes += (G::WE + G::WT) * sizeof(T);
    if (need_x) bytes += G::WT * sizeof(T);
    mbar_arrive_expect_tx(&bar[slot], bytes);
    if (!(skip_first && m == mlo)) bulk_g2s(sl + G::OFF_S, src + rowoff + i0 - G::H, G::WS * sizeof(T), &bar[slot]);
    if (need_d) bulk_g2s(sl + G::OFF_D, dold + rowoff + i0 - G::H, G::WS * sizeof(T), &bar[slot]);
    if (need_n) bulk_g2s(sl + G::OFF_N, gd.cn + rowoff + i0, G::WT * sizeof(T), &bar[slot]);
    if (need_row) {
      bulk_g2s(sl + G::OFF_E, gd.ce + rowoff + i0 - G::H, G::WE * sizeof(T), &bar[slot]);
      bulk_g2s(sl + G::OFF_A, gd.a + rowoff + i0, G::WT * sizeof(T), &bar[slot]);
    }
    if (need_x) bulk_g2s(sl + G::OFF_X, xb + rowoff + i0, G::WT * sizeof(T), &bar[slot]);
  };

  if (tid == 0) {
    for (int s = 0; s < G::NST; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int issued = min(mhi, mlo + G::NST - 1);   // last row handed to the copy engine (thread 0)
  if (tid == 0) {
    for (int m = mlo; m <= issued; ++m) issue(m);
  }

  double acc0 = 0.0, acc1 = 0.0;
  bool ok = true;
  int failed_at = mhi + 1;
  for (int m = mlo; m <= mhi; ++m) {
    const int slot = (m - mlo) % G::NST;
    const uint32_t parity = (uint32_t)(((m - mlo) / G::NST) & 1);
    const bool got = mbar_wait_bounded(&bar[slot], parity, p.timeout_ns);
    if (!__syncthreads_and(got)) { ok = false; failed_at = m; break; }
    const T *sl = ring + (size_t)slot * G::SLOT;
    T *dnm = dn + (size_t)((m + 6) % 3) * G::WDN;
    // d' on row m over columns [i0-1, i0+TX+1)
    for (int c = tid; c < G::WDN; c += TX) {
      const int k = c - 1 + G::H;
      T v = sl[G::OFF_S + k];
      if (kind == K1_ITER) v = fma(beta, sl[G::OFF_D + k], v);
      dnm[c] = v;
    }
    __syncthreads();
    const int r = m - 1;
    if (r >= j0) {
      const int col = i0 + tid;
      if (col < nx) {
        const T *slr = ring + (size_t)((r - mlo) % G::NST) * G::SLOT;
        const T *sls = ring + (size_t)((r - 1 - mlo) % G::NST) * G::SLOT;
        const T *dr = dn + (size_t)((r + 6) % 3) * G::WDN;
        const T *ds = dn + (size_t)((r - 1 + 6) % 3) * G::WDN;
        const T c_ctr = dr[tid + 1];
        T av = -sls[G::OFF_N + tid] * ds[tid + 1];
        av = fma(-slr[G::OFF_E + G::H + tid - 1], dr[tid], av);
        av = fma(slr[G::OFF_A + tid], c_ctr, av);
        av = fma(-slr[G::OFF_E + G::H + tid], dr[tid + 2], av);
        av = fma(-slr[G::OFF_N + tid], dnm[tid + 1], av);
        const size_t ro = (size_t)r * pitch;
        if (kind == K1_ITER) {
          const T xv = fma(pend, slr[G::OFF_D + G::H + tid], slr[G::OFF_X + tid]);
          store_dup(gd.d[dsel ^ 1] + ro, col, nx, c_ctr);
          store_dup(gd.x + ro, col, nx, xv);
          store_dup(gd.q + ro, col, nx, av);
          acc0 = fma((double)c_ctr, (double)av, acc0);
        } else if (kind == K1_SPMV) {
          store_dup(gd.q + ro, col, nx, av);
        } else {
          const T bv = slr[G::OFF_X + tid];
          const T rv = bv - av;
          store_dup(gd.r[rsel1] + ro, col, nx, rv);
          acc0 = fma((double)rv, (double)rv, acc0);
          acc1 = fma((double)bv, (double)bv, acc1);
        }
      }
    }
    __syncthreads();
    // the slot of row m-2 is free: refill it with row m-2+NST
    if (tid == 0 && m - 2 >= mlo) {
      const int nm = m - 2 + G::NST;
      if (nm <= mhi) { fence_proxy_async(); issue(nm); issued = nm; }
    }
  }
  if (!ok && tid == 0) {
    // give up: record it, and wait (bounded) for the copies still in flight
    flag_timeout(st);
    for (int m = failed_at; m <= issued; ++m)
      mbar_wait_bounded(&bar[(m - mlo) % G::NST], (uint32_t)(((m - mlo) / G::NST) & 1), p.timeout_ns);
  }
  if (kind == K1_SPMV) return;
  if (grid_reduce2<TX>(acc0, acc1, gd.partial, un.u, gd.n_units, &st->cnt1, red, flag)) {
    if (threadIdx.x == 0) {
      if (kind == K1_ITER) {
        const double dq = acc0;
        st->dq = dq;
        st->pending = 0.0;
        st->dsel = dsel ^ 1;
        if (st->status != PCG_OK) grid_finished(st, ls, PCG_OK, false, p);
        else if (!(dq > 0.0) || !isfinite(dq)) grid_finished(st, ls, PCG_EBREAKDOWN, false, p);
        else st->alpha = st->rho / dq;
      } else if (kind == K1_RESID_INIT) {
        st->rr = acc0;
        st->bb = acc1;
        if (st->status != PCG_OK) grid_finished(st, ls, PCG_OK, false, p);
        else if (!isfinite(acc1) || !isfinite(acc0)) grid_finished(st, ls, PCG_EBREAKDOWN, false, p);
        else if (acc1 == 0.0) { st->bzero = 1; grid_finished(st, ls, PCG_OK, false, p); }
      } else {
        st->rr_true = acc0;
      }
    }
  }
}

// ------------------------------------------------------------ kernel 2
// Preconditioner pass (Algorithm 1, line 7): r' = r - alpha q;
// s = Z (D^-1 (Z^T r')); sums s.r' and r'.r'. Kinds: K2_ITER, K2_INIT
// (alpha = 0, q not read), K2_APPLY (s = M^-1 r only, r in r[0]).
template <typename T, int TX, class P>
struct K2Geom {
  static constexpr int AL = 16 / (int)sizeof(T);
  static constexpr int R = P::R, LD = P::LD, NZ = P::NZ;
  static constexpr int HR = round_up_c(2 * R, AL);   // halo of r, q
  static constexpr int HZ = round_up_c(R, AL);       // halo of Z planes and D^-1
  static constexpr int WR = TX + 2 * HR, WZ = TX + 2 * HZ;
  static constexpr int WRC = TX + 4 * R;             // r' computed on [i0-2R, i0+TX+2R)
  static constexpr int WTC = TX + 2 * R;             // t computed on [i0-R, i0+TX+R)
  static constexpr int RING = LD + 1;                // rows of r' and of t kept
  static constexpr int NST = LD + 1 + 3;             // ring slots
  static constexpr int OFF_R = 0, OFF_Q = WR, OFF_Z = 2 * WR, OFF_DI = 2 * WR + NZ * WZ, SLOT = OFF_DI + WZ;
  static constexpr size_t SMEM =
      128 + sizeof(T) * ((size_t)NST * SLOT + (size_t)RING * WRC + (size_t)RING * WTC) + 16 * 2 * (TX / 32) + 64;
};

template <typename T, int TX, class P>
__global__ void __launch_bounds__(TX) k_precond(KParams p) {
  using G = K2Geom<T, TX, P>;
  constexpr int R = P::R, LD = P::LD, NZ = P::NZ, NW = P::NW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
  T *ring = reinterpret_cast<T *>(smem_raw + 128);
  T *rn = ring + (size_t)G::NST * G::SLOT;
  T *tt = rn + (size_t)G::RING * G::WRC;
  double *red = reinterpret_cast<double *>(tt + (size_t)G::RING * G::WTC);
  int *flag = reinterpret_cast<int *>(red + 2 * (TX / 32));

  const Unit un = p.units[blockIdx.x];
  const GridDev<T> &gd = reinterpret_cast<const GridDev<T> *>(p.grids)[un.g];
  SolveState *st = gd.st;
  LaunchState *ls = p.ls;
  const int kind = p.kind;

  if (kind == K2_ITER && p.use_cond && *(volatile int32_t *)&ls->stop) return;
  if (kind != K2_APPLY && *(volatile int32_t *)&st->done) return;

  const int nx = gd.nx, ny = gd.ny, pitch = gd.pitch;
  const int i0 = un.sx * TX, j0 = un.sy * gd.ty;
  const int rend = min(j0 + gd.ty, ny);
  const int mlo = j0 - LD, mhi = rend + LD - 1;
  const int tid = threadIdx.x;
  const T alpha = (kind == K2_ITER) ? (T)st->alpha : (T)0;
  const int rsel = (kind == K2_APPLY) ? 0 : st->rsel;
  const T *rin = gd.r[rsel];
  T *rout = gd.r[rsel ^ 1];
  const bool skip_first = (p.dbg_skip_unit == (int)blockIdx.x);

  auto issue = [&](int m) {
    const int slot = (m - mlo) % G::NST;
    T *sl = ring + (size_t)slot * G::SLOT;
    const size_t rowoff = (size_t)m * pitch;
    const bool need_q = (kind == K2_ITER);
    const bool need_z = (m >= j0);
    uint32_t bytes = G::WR * sizeof(T);
    if (need_q) bytes += G::WR * sizeof(T);
    if (need_z) bytes += (NZ + 1) * G::WZ * sizeof(T);
    mbar_arrive_expect_tx(&bar[slot], bytes);
    if (!(skip_first && m == mlo)) bulk_g2s(sl + G::OFF_R, rin + rowoff + i0 - G::HR, G::WR * sizeof(T), &bar[slot]);
    if (need_q) bulk_g2s(sl + G::OFF_Q, gd.q + rowoff + i0 - G::HR, G::WR * sizeof(T), &bar[slot]);
    if (need_z) {
#pragma unroll
      for (int s = 0; s < NZ; ++s)
        bulk_g2s(sl + G::OFF_Z + s * G::WZ, gd.z[s] + rowoff + i0 - G::HZ, G::WZ * sizeof(T), &bar[slot]);
      bulk_g2s(sl + G::OFF_DI, gd.dinv + rowoff + i0 - G::HZ, G::WZ * sizeof(T), &bar[slot]);
    }
  };

  if (tid == 0) {
    for (int s = 0; s < G::NST; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int issued = min(mhi, mlo + G::NST - 1);
  if (tid == 0) {
    for (int m = mlo; m <= issued; ++m) issue(m);
  }

  double acc0 = 0.0, acc1 = 0.0;
  bool ok = true;
  int failed_at = mhi + 1;
  for (int m = mlo; m <= mhi; ++m) {
    const int slot = (m - mlo) % G::NST;
    const uint32_t parity = (uint32_t)(((m - mlo) / G::NST) & 1);
    const bool got = mbar_wait_bounded(&bar[slot], parity, p.timeout_ns);
    if (!__syncthreads_and(got)) { ok = false; failed_at = m; break; }
    const T *sl = ring + (size_t)slot * G::SLOT;
    // r' on row m over [i0-2R, i0+TX+2R)
    T *rnm = rn + (size_t)((m + 8) % G::RING) * G::WRC;
    for (int c = tid; c < G::WRC; c += TX) {
      const int k = c + G::HR - 2 * R;
      T v = sl[G::OFF_R + k];
      if (kind == K2_ITER) v = fma(-alpha, sl[G::OFF_Q + k], v);
      rnm[c] = v;
    }
    __syncthreads();
    // t = D^-1 (Z^T r') on row m over [i0-R, i0+TX+R)
    if (m >= j0) {
      T *tm = tt + (size_t)((m + 8) % G::RING) * G::WTC;
      for (int c = tid; c < G::WTC; c += TX) {
        T acc = (T)0;
        if (m < ny) {
          const int kz = c + G::HZ - R;
          acc = rnm[c + R];
#pragma unroll
          for (int s = 0; s < NZ; ++s) {
            const T *rrow = rn + (size_t)((m + P::dy(s) + 8) % G::RING) * G::WRC;
            acc = fma(sl[G::OFF_Z + s * G::WZ + kz], rrow[c + R + P::dx(s)], acc);
          }
          if (NW > 0) {
            const int col = i0 - R + c;
            const int cm = ((col % nx) + nx) % nx;
#pragma unroll
            for (int w = 0; w < (NW > 0 ? NW : 1); ++w)
              if (cm == nx - 1 - P::wcol(w)) acc = fma(gd.zwrap[(size_t)m * NW + w], rnm[c + R + P::wdx(w)], acc);
          }
          acc *= sl[G::OFF_DI + kz];
        }
        tm[c] = acc;
      }
    }
    __syncthreads();
    // s = Z t on row r = m - LD
    const int r = m - LD;
    if (r >= j0) {
      const int col = i0 + tid;
      if (col < nx) {
        const T *tr = tt + (size_t)((r + 8) % G::RING) * G::WTC;
        T acc = tr[tid + R];
#pragma unroll
        for (int s = 0; s < NZ; ++s) {
          const int rowz = r - P::dy(s);           // row of the column holding Z[(col,r), that column]
          const T *slz = ring + (size_t)((rowz - mlo) % G::NST) * G::SLOT;
          const T *trow = tt + (size_t)((rowz + 8) % G::RING) * G::WTC;
          acc = fma(slz[G::OFF_Z + s * G::WZ + tid - P::dx(s) + G::HZ], trow[tid + R - P::dx(s)], acc);
        }
        if (NW > 0) {
#pragma unroll
          for (int w = 0; w < (NW > 0 ? NW : 1); ++w) {
            const int target = ((P::wdx(w) - 1 - P::wcol(w)) % nx + nx) % nx;
            if (col == target) acc = fma(gd.zwrap[(size_t)r * NW + w], tr[tid + R - P::wdx(w)], acc);
          }
        }
        const T *rnr = rn + (size_t)((r + 8) % G::RING) * G::WRC;
        const T rv = rnr[tid + 2 * R];
        const size_t ro = (size_t)r * pitch;
        store_dup(gd.s + ro, col, nx, acc);
        if (kind != K2_APPLY) store_dup(rout + ro, col, nx, rv);
        acc0 = fma((double)acc, (double)rv, acc0);
        acc1 = fma((double)rv, (double)rv, acc1);
      }
    }
    __syncthreads();
    if (tid == 0 && m - LD >= mlo) {
      const int nm = m - LD + G::NST;
      if (nm <= mhi) { fence_proxy_async(); issue(nm); issued = nm; }
    }
  }
  if (!ok && tid == 0) {
    flag_timeout(st);
    for (int m = failed_at; m <= issued; ++m)
      mbar_wait_bounded(&bar[(m - mlo) % G::NST], (uint32_t)(((m - mlo) / G::NST) & 1), p.timeout_ns);
  }
  if (kind == K2_APPLY) return;
  if (grid_reduce2<TX>(acc0, acc1, gd.partial, un.u, gd.n_units, &st->cnt2, red, flag)) {
    if (threadIdx.x == 0) {
      const double rho_new = acc0, rr = acc1;
      st->rr = rr;
      st->rsel = rsel ^ 1;
      if (kind == K2_ITER) {
        st->beta = rho_new / st->rho;
        st->pending = st->alpha;
        st->iter += 1;
      } else {
        st->beta = 0.0;
        st->pending = 0.0;
      }
      st->rho = rho_new;
      const double relres = sqrt(rr) / sqrt(st->bb);
      if (st->status != PCG_OK) grid_finished(st, ls, PCG_OK, true, p);
      else if (!isfinite(rho_new) || !isfinite(rr)) grid_finished(st, ls, PCG_EBREAKDOWN, true, p);
      else if (!(relres > st->rtol)) grid_finished(st, ls, PCG_OK, true, p);
      else if (st->iter >= st->max_iter) grid_finished(st, ls, PCG_ENOTCONV, true, p);
      else if (!(rho_new > 0.0)) grid_finished(st, ls, PCG_EBREAKDOWN, true, p);
    }
  }
}

// ------------------------------------------------------------ small kernels
// x += pending * d (the last step's update), or x = 0 when b = 0.
template <typename T, int TX>
__global__ void __launch_bounds__(TX) k_finalize(KParams p) {
  const Unit un = p.units[blockIdx.x];
  const GridDev<T> &gd = reinterpret_cast<const GridDev<T> *>(p.grids)[un.g];
  SolveState *st = gd.st;
  if (*(volatile int32_t *)&st->retired) return;
  const int col = un.sx * TX + threadIdx.x;
  const int j0 = un.sy * gd.ty, rend = min(j0 + gd.ty, gd.ny);
  const T pend = (T)st->pending;
  const bool zero = st->bzero != 0;
  const T *d = gd.d[st->dsel];
  if (col < gd.nx) {
    for (int r = j0; r < rend; ++r) {
      const size_t ro = (size_t)r * gd.pitch;
      T xv = zero ? (T)0 : fma(pend, d[ro + col], gd.x[ro + col]);
      store_dup(gd.x + ro, col, gd.nx, xv);
    }
  }
}

// user [ny][nx] -> padded plane (zero on land), with periodic copies
template <typename T, typename U, int TX>
__global__ void __launch_bounds__(TX) k_pack(KParams p, const U *user, int which) {
  const Unit un = p.units[blockIdx.x];
  const GridDev<T> &gd = reinterpret_cast<const GridDev<T> *>(p.grids)[un.g];
  T *dst = which == 0 ? const_cast<T *>(gd.b) : which == 1 ? gd.x : which == 2 ? gd.r[0] : gd.d[0];
  const int col = un.sx * TX + threadIdx.x;
  const int j0 = un.sy * gd.ty, rend = min(j0 + gd.ty, gd.ny);
  if (col < gd.nx) {
    for (int r = j0; r < rend; ++r) {
      const size_t ro = (size_t)r * gd.pitch;
      const T v = gd.a[ro + col] > (T)0 ? (T)user[(size_t)r * gd.nx + col] : (T)0;
      store_dup(dst + ro, col, gd.nx, v);
    }
  }
}

// padded plane -> user [ny][nx] (land = 0), over every cell
template <typename T, typename U>
__global__ void k_unpack(const GridDev<T> *gdp, U *user, int which) {
  const GridDev<T> &gd = *gdp;
  const T *srcp = which == 0 ? gd.x : which == 1 ? gd.s : which == 2 ? gd.q : gd.r[0];
  const size_t n = (size_t)gd.nx * gd.ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / gd.nx), i = (int)(e % gd.nx);
    const size_t o = (size_t)j * gd.pitch + i;
    user[e] = gd.a[o] > (T)0 ? (U)srcp[o] : (U)0;
  }
}

}  // namespace pcg
