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
__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

// Exact widening of binary32 to binary64 with integer operations only (IEEE
// 754 formats: sign kept; exponent re-biased by 1023 - 127; the 23-bit
// fraction moved to the top of the 52-bit fraction; subnormals normalised by a
// leading-zero count; infinities and NaNs keep their fraction bits). On this
// GPU the hardware conversion runs on the slow FP64 pipe, which the binary32
// kernels must leave alone.
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t sgn = u & 0x80000000u, e = (u >> 23) & 0xFFu;
  uint32_t f = u & 0x7FFFFFu, E;
  if (e == 0xFFu) {
    E = 0x7FFu;
  } else if (e != 0u) {
    E = e + (1023u - 127u);
  } else if (f == 0u) {
    E = 0u;
  } else {
    const uint32_t top = 31u - (uint32_t)__clz((int)f);   // bit of the leading one, < 23
    E = top + 874u;                                         // value = f * 2^-149
    f = (f << (23u - top)) & 0x7FFFFFu;
  }
  return __hiloint2double((int)(sgn | (E << 20) | (f >> 3)), (int)(f << 29));
}

// Dot-product term accumulation. binary64 kernels accumulate in binary64.
// binary32 kernels keep a binary32 partial sum per thread over the rows of
// its column in one work unit (at most a unit's height of terms); the partial
// is widened exactly and added into the binary64 accumulator when the unit is
// done, so every long accumulation is in binary64.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double total() const { return v; }
};
template <>
struct DotAcc<float> {
  float v = 0.0f;
  __device__ __forceinline__ void add(float a, float b) { v = fmaf(a, b, v); }
  __device__ __forceinline__ double total() const { return to_f64(v); }
};

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

// End the conditional loop graph after the current body: exactly one thread
// per graph launch sets the condition (concurrent settings are not allowed).
__device__ __forceinline__ void clear_loop_condition(LaunchState *ls, const KParams &p) {
  if (p.use_cond && atomicExch(&ls->cond_cleared, 1) == 0) cudaGraphSetConditional(ls->cond, 0);
}

__device__ __forceinline__ void grid_finished(SolveState *st, LaunchState *ls, int status, bool may_set_cond,
                                             const KParams &p) {
  if (status != PCG_OK) atomicCAS(&st->status, PCG_OK, status);
  st->done = 1;
  __threadfence();
  const int prev = atomicSub(&ls->active, 1);
  if (prev == 1 && may_set_cond) clear_loop_condition(ls, p);
}

// Loop guard, run by one thread of the first preconditioner launch of each
// loop body (the body's last kernel, so a body always runs whole): counts the
// bodies and ends the loop once all grids are done, after max_launches
// bodies, or when the wall-clock budget is spent.
__device__ __forceinline__ void loop_guard(LaunchState *ls, const KParams &p) {
  const int l = atomicAdd(&ls->launches, 1) + 1;
  const uint64_t now = global_ns();
  if (ls->t0_ns == 0) ls->t0_ns = now;
  const bool late = now - ls->t0_ns > ls->budget_ns;
  if (late) ls->timed_out = 1;
  if (l >= ls->max_launches || late) ls->stop = 1;
  if (l >= ls->max_launches || late || atomicAdd(&ls->active, 0) == 0) clear_loop_condition(ls, p);
}

__device__ __forceinline__ void flag_timeout(SolveState *st) { atomicCAS(&st->status, PCG_OK, PCG_ETIMEOUT); }

// ------------------------------------------------------------ row streaming
// A CTA is TX compute threads plus one producer warp. The producer streams
// rows: lane a owns field a of a row (source plane, place in a ring slot,
// size) and issues its bulk copy (cp.async.bulk) into the slot; lane 0 first
// arms the slot's "full" mbarrier with the row's byte count. A bulk copy
// occupies its issuing thread for several hundred ns on this GPU, so the
// producer runs ahead on its own and the compute threads never wait for an
// issue, only for data. When the compute threads are done with a row, one of
// them arrives on the slot's "empty" mbarrier; the producer waits for that
// before it refills the slot.
struct RowCopy {
  const char *src;             // element (i0 - halo, row 0) of the plane, as bytes
  uint32_t dst;                // byte offset inside a ring slot
  uint32_t bytes;
  int when;                    // 0: every streamed row; 1: rows < mhi; 2: rows in [j0, mhi); 3: rows >= j0
};

__device__ __forceinline__ bool row_wanted(int when, int m, int j0, int mhi) {
  switch (when) {
    case 1: return m < mhi;
    case 2: return m >= j0 && m < mhi;
    case 3: return m >= j0;
    default: return true;
  }
}

// Issue row m into its slot (producer warp, all lanes).
__device__ __forceinline__ void issue_row(const RowCopy &c, unsigned char *slot_base, uint64_t *full, int m,
                                          size_t pitch_bytes, int j0, int mhi, bool skip) {
  const bool want = c.src && row_wanted(c.when, m, j0, mhi);
  const uint32_t total = __reduce_add_sync(0xffffffffu, want ? c.bytes : 0u);
  if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(full, total);
  __syncwarp();
  if (want && !skip) {
    fence_proxy_async();
    bulk_g2s(slot_base + c.dst, c.src + (ptrdiff_t)m * (ptrdiff_t)pitch_bytes, c.bytes, full);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Barrier of the NT compute threads only (named barrier 1), with an AND vote.
template <int NT>
__device__ __forceinline__ bool compute_sync_and(bool v) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.cta.red.and.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(NT)
      : "memory");
  return out != 0;
}

// The producer loop: rows [mlo, mhi] into NST ring slots; producer warp w of
// P handles rows mlo + w, mlo + w + P, ... (a bulk copy blocks its issuing
// thread for several hundred ns, so several warps issue side by side). Slot
// of row n is (n - mlo) % NST; its k-th fill waits for the (k-1)-th release.
// Returns the last row issued. Bounded: a release that never comes ends the
// loop.
template <int NST>
__device__ __forceinline__ int produce_rows(const RowCopy &c, unsigned char *ring, int slot_bytes, uint64_t *full,
                                            uint64_t *empty, int mlo, int mhi, size_t pitch_bytes, int j0,
                                            bool skip_first, uint64_t timeout_ns, const volatile int *abort,
                                            int first, int stride) {
  int last = mlo - 1;
  for (int n = mlo + first; n <= mhi; n += stride) {
    const int slot = (NST & (NST - 1)) == 0 ? ((n - mlo) & (NST - 1)) : ((n - mlo) % NST), fill = (n - mlo) / NST;
    if (fill > 0) {
      bool ok = true;
      if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(&empty[slot], (uint32_t)((fill - 1) & 1), timeout_ns);
      ok = __shfl_sync(0xffffffffu, ok, 0) && !*abort;
      if (!ok) break;
    }
    issue_row(c, ring + (size_t)slot * slot_bytes, &full[slot], n, pitch_bytes, j0, mhi, skip_first && n == mlo);
    last = n;
  }
  return last;
}

// ------------------------------------------------------------ kernel 1
// Stencil pass (Section 3, Eq. 9 in SPD form). Kinds:
//  K1_ITER        d' = s + beta d; x += pending d; q = A d'; sum d'.q
//  K1_RESID_INIT  r = b - A x; sums r.r and b.b
//  K1_RESID_CHECK r = b - A x; sum r.r (true residual)
//  K1_SPMV        q = A v (v in d[0])
// Step m computes d' on row m, then q on row m - 2 (whose north neighbour
// row m - 1 was finished in the previous step): one compute barrier per row.
template <typename T, int TX>
struct K1Geom {
  static constexpr int AL = 16 / (int)sizeof(T);     // elements per 16 bytes
  static constexpr int H = AL;                       // halo of the centre fields (>= 1)
  static constexpr int WS = TX + 2 * H;              // s, d_old / x / v: [i0-H, i0+TX+H)
  static constexpr int WE = TX + H;                  // c_e: [i0-H, i0+TX)
  static constexpr int WT = TX;                      // c_n, a, x / b
  static constexpr int NST = 8;                      // ring slots (a power of two): rows m-3..m live, 4 ahead
  static constexpr int NDN = 4;                      // rows of d' kept (a power of two)
  static constexpr int NPW = 1;                      // producer warps
  static constexpr int NT = TX + 32 * NPW;           // compute threads + producer warps
  static constexpr int OFF_S = 0, OFF_D = WS, OFF_E = 2 * WS, OFF_N = 2 * WS + WE, OFF_A = OFF_N + WT,
                       OFF_X = OFF_A + WT, SLOT = OFF_X + WT;
  static constexpr int WDN = TX + 2;                 // d' ring: [i0-1, i0+TX+1)
  static constexpr size_t SMEM = 256 + sizeof(T) * ((size_t)NST * SLOT + NDN * WDN) + 16 * (NT / 32) + 64;
  static_assert(2 * NST * 8 <= 224 && 3 + NPW <= 8, "barrier / control area of the first 256 bytes");
};

template <typename T, int TX>
__global__ void __launch_bounds__(TX + 32 * K1Geom<T, TX>::NPW) k_stencil(KParams p) {
  using G = K1Geom<T, TX>;
  constexpr int NT = G::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
  uint64_t *empty = full + G::NST;
  volatile int *ctl = reinterpret_cast<volatile int *>(smem_raw + 224);   // abort, -, consumed, last row per producer
  unsigned char *ring_b = smem_raw + 256;
  const T *ring = reinterpret_cast<const T *>(ring_b);
  T *dn = reinterpret_cast<T *>(ring_b + sizeof(T) * (size_t)G::NST * G::SLOT);
  double *red = reinterpret_cast<double *>(dn + (size_t)G::NDN * G::WDN);
  int *flag = reinterpret_cast<int *>(red + 2 * (NT / 32));

  const Unit un = p.units[blockIdx.x];
  const GridDev<T> *gdp = reinterpret_cast<const GridDev<T> *>(p.grids) + un.g;
  SolveState *st = gdp->st;
  LaunchState *ls = p.ls;
  const int kind = p.kind;
  const int tid = threadIdx.x;

  if ((kind == K1_ITER || kind == K1_RESID_INIT) && *(volatile int32_t *)&st->done) return;
  if (kind == K1_RESID_CHECK && *(volatile int32_t *)&st->retired) return;

  const int nx = gdp->nx, ny = gdp->ny, pitch = gdp->pitch, ty = gdp->ty;
  const int i0 = un.sx * TX, j0 = un.sy * ty;
  const int rend = min(j0 + ty, ny);
  const int mlo = j0 - 1, mhi = rend;          // rows streamed: south halo row .. north look-ahead row
  const int dsel = st->dsel, rsel = st->rsel;
  const size_t pitch_b = (size_t)pitch * sizeof(T);
  constexpr int SLOTB = G::SLOT * (int)sizeof(T);

  if (tid == 0) {
    for (int s = 0; s < G::NST; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    ctl[0] = 0; ctl[1] = mlo - 1; ctl[2] = mlo - 1;
    for (int w = 0; w < G::NPW; ++w) ctl[3 + w] = mlo - 1;
    fence_mbar_init();
  }
  __syncthreads();

  double acc0 = 0.0, acc1 = 0.0;
  DotAcc<T> dot0, dot1;
  if (tid >= TX) {
    // ---- producer warps
    const int lane = (tid - TX) & 31, pw = (tid - TX) >> 5;
    RowCopy c{nullptr, 0, 0, 0};
    const T *src = (kind == K1_ITER) ? gdp->s : (kind == K1_SPMV) ? gdp->d[0] : gdp->x;
    auto at = [&](const T *plane, int col) { return reinterpret_cast<const char *>(plane + i0 + col); };
    switch (lane) {
      case 0: c = RowCopy{at(src, -G::H), (uint32_t)(G::OFF_S * sizeof(T)), (uint32_t)(G::WS * sizeof(T)), 0}; break;
      case 1: if (kind == K1_ITER) c = RowCopy{at(gdp->d[dsel], -G::H), (uint32_t)(G::OFF_D * sizeof(T)), (uint32_t)(G::WS * sizeof(T)), 0}; break;
      case 2: c = RowCopy{at(gdp->cn, 0), (uint32_t)(G::OFF_N * sizeof(T)), (uint32_t)(G::WT * sizeof(T)), 1}; break;
      case 3: c = RowCopy{at(gdp->ce, -G::H), (uint32_t)(G::OFF_E * sizeof(T)), (uint32_t)(G::WE * sizeof(T)), 2}; break;
      case 4: c = RowCopy{at(gdp->a, 0), (uint32_t)(G::OFF_A * sizeof(T)), (uint32_t)(G::WT * sizeof(T)), 2}; break;
      case 5: if (kind != K1_SPMV) c = RowCopy{at(kind == K1_ITER ? gdp->x : gdp->b, 0), (uint32_t)(G::OFF_X * sizeof(T)), (uint32_t)(G::WT * sizeof(T)), 2}; break;
      default: break;
    }
    const bool skip_first = (p.dbg_skip_unit == (int)blockIdx.x) && lane == 0 && pw == 0;
    const int last = produce_rows<G::NST>(c, ring_b, SLOTB, full, empty, mlo, mhi, pitch_b, j0, skip_first,
                                          p.timeout_ns, ctl, pw, G::NPW);
    if (lane == 0) ctl[3 + pw] = last;
  } else {
    // ---- compute threads
    const T beta = (kind == K1_ITER) ? (T)st->beta : (T)0;
    const T pend = (kind == K1_ITER) ? (T)st->pending : (T)0;
    T *const d_out = gdp->d[dsel ^ 1];
    T *const x_out = gdp->x;
    T *const q_out = gdp->q;
    T *const r_out = gdp->r[rsel];
    int consumed = mlo - 1;
    for (int m = mlo; m <= mhi + 1; ++m) {
      bool got = true;
      if (m <= mhi) {
        const int slot = (m - mlo) & (G::NST - 1);
        got = mbar_wait_bounded(&full[slot], (uint32_t)(((m - mlo) / G::NST) & 1), p.timeout_ns);
        const T *sl = ring + (size_t)slot * G::SLOT;
        T *dnm = dn + (size_t)((m + 8) & (G::NDN - 1)) * G::WDN;
        // d' on row m over columns [i0-1, i0+TX+1)
        for (int c = tid; c < G::WDN; c += TX) {
          const int k = c - 1 + G::H;
          T v = sl[G::OFF_S + k];
          if (kind == K1_ITER) v = fma(beta, sl[G::OFF_D + k], v);
          dnm[c] = v;
        }
      }
      const int r = m - 2;
      if (r >= j0 && r < rend) {
        const int col = i0 + tid;
        if (col < nx) {
          const T *slr = ring + (size_t)((r - mlo) & (G::NST - 1)) * G::SLOT;
          const T *sls = ring + (size_t)((r - 1 - mlo) & (G::NST - 1)) * G::SLOT;
          const T *dr = dn + (size_t)((r + 8) & (G::NDN - 1)) * G::WDN;
          const T *ds = dn + (size_t)((r - 1 + 8) & (G::NDN - 1)) * G::WDN;
          const T *dnn = dn + (size_t)((r + 1 + 8) & (G::NDN - 1)) * G::WDN;
          const T c_ctr = dr[tid + 1];
          T av = -sls[G::OFF_N + tid] * ds[tid + 1];
          av = fma(-slr[G::OFF_E + G::H + tid - 1], dr[tid], av);
          av = fma(slr[G::OFF_A + tid], c_ctr, av);
          av = fma(-slr[G::OFF_E + G::H + tid], dr[tid + 2], av);
          av = fma(-slr[G::OFF_N + tid], dnn[tid + 1], av);
          const size_t ro = (size_t)r * pitch;
          if (kind == K1_ITER) {
            const T xv = fma(pend, slr[G::OFF_D + G::H + tid], slr[G::OFF_X + tid]);
            store_dup(d_out + ro, col, nx, c_ctr);
            store_dup(x_out + ro, col, nx, xv);
            store_dup(q_out + ro, col, nx, av);
            dot0.add(c_ctr, av);
          } else if (kind == K1_SPMV) {
            store_dup(q_out + ro, col, nx, av);
          } else {
            const T bv = slr[G::OFF_X + tid];
            const T rv = bv - av;
            store_dup(r_out + ro, col, nx, rv);
            dot0.add(rv, rv);
            dot1.add(bv, bv);
          }
        }
      }
      if (!compute_sync_and<TX>(got)) {
        if (tid == 0) { ctl[0] = 1; flag_timeout(st); }
        break;
      }
      if (m <= mhi) consumed = m;
      // row m-3 is finished: its slot may be refilled
      if (tid == 0 && m - 3 >= mlo && m - 3 + G::NST <= mhi) mbar_arrive(&empty[(m - 3 - mlo) & (G::NST - 1)]);
    }
    if (tid == 0) ctl[2] = consumed;
    acc0 = dot0.total();
    acc1 = dot1.total();
  }
  __syncthreads();
  if (tid == 0 && ctl[0]) {
    // the compute threads gave up: wait (bounded) for the rows still in flight
    for (int w = 0; w < G::NPW; ++w)
      for (int m = mlo + w; m <= ctl[3 + w]; m += G::NPW)
        if (m > ctl[2])
          mbar_wait_bounded(&full[(m - mlo) & (G::NST - 1)], (uint32_t)(((m - mlo) / G::NST) & 1), p.timeout_ns);
  }
  if (kind == K1_SPMV) return;
  if (grid_reduce2<NT>(acc0, acc1, gdp->partial, un.u, gdp->n_units, &st->cnt1, red, flag)) {
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
// Preconditioner pass (the residual update and preconditioning step of
// Algorithm 1): r' = r - alpha q; s = Z (D^-1 (Z^T r')); sums s.r' and r'.r'.
// Kinds: K2_ITER, K2_INIT (alpha = 0, q not read), K2_APPLY (s = M^-1 r only,
// r in r[0]). Step m computes r' on row m, t = D^-1 Z^T r' on row m - 1 (Z^T
// pulls from rows m-1-LD..m-1, finished before) and s = Z t on row m - 2 - LD
// (Z pushes from rows up to m - 2): one compute barrier per row.
template <typename T, int TX, class P>
struct K2Geom {
  static constexpr int AL = 16 / (int)sizeof(T);
  static constexpr int R = P::R, LD = P::LD, NZ = P::NZ;
  static constexpr int HR = round_up_c(2 * R, AL);   // halo of r, q
  static constexpr int HZ = round_up_c(R, AL);       // halo of Z planes and D^-1
  static constexpr int WR = TX + 2 * HR, WZ = TX + 2 * HZ;
  static constexpr int WRC = TX + 4 * R;             // r' computed on [i0-2R, i0+TX+2R)
  static constexpr int WTC = TX + 2 * R;             // t computed on [i0-R, i0+TX+R)
  static constexpr int NRN = pow2_at_least(LD + 3);  // rows of r' kept (m-2-LD .. m)
  static constexpr int NTT = pow2_at_least(LD + 2);  // rows of t kept (m-2-LD .. m-1)
  // rows streamed ahead: binary64 is bound by the FP64 pipe, so shared memory
  // goes to CTAs (latency hiding for the FP64 work); binary32 is bound by
  // HBM, so it goes to rows in flight
  // ring slots: rows m-2-LD .. m live plus rows in flight. binary64 is bound
  // by the FP64 pipe, so its shared memory goes to CTAs (one row ahead);
  // binary32 is bound by HBM, so it keeps more rows in flight.
  static constexpr int NST = sizeof(T) == 8 ? LD + 4 : pow2_at_least(LD + 5);
  __device__ static constexpr int slot(int x) { return (NST & (NST - 1)) == 0 ? (x & (NST - 1)) : (x % NST); }
  static constexpr int NPW = 1;                      // producer warps
  static constexpr int NT = TX + 32 * NPW;           // compute threads + producer warps
  static constexpr int OFF_R = 0, OFF_Q = WR, OFF_Z = 2 * WR, OFF_DI = 2 * WR + NZ * WZ, SLOT = OFF_DI + WZ;
  static constexpr size_t SMEM =
      256 + sizeof(T) * ((size_t)NST * SLOT + (size_t)NRN * WRC + (size_t)NTT * WTC) + 16 * (NT / 32) + 64;
  static_assert(2 * NST * 8 <= 224 && 3 + NPW <= 8, "barrier / control area of the first 256 bytes");
};

template <typename T, int TX, class P>
__global__ void __launch_bounds__(TX + 32 * K2Geom<T, TX, P>::NPW) k_precond(KParams p) {
  using G = K2Geom<T, TX, P>;
  constexpr int R = P::R, LD = P::LD, NZ = P::NZ, NW = P::NW, NT = G::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
  uint64_t *empty = full + G::NST;
  volatile int *ctl = reinterpret_cast<volatile int *>(smem_raw + 224);
  unsigned char *ring_b = smem_raw + 256;
  const T *ring = reinterpret_cast<const T *>(ring_b);
  T *rn = reinterpret_cast<T *>(ring_b + sizeof(T) * (size_t)G::NST * G::SLOT);
  T *tt = rn + (size_t)G::NRN * G::WRC;
  double *red = reinterpret_cast<double *>(tt + (size_t)G::NTT * G::WTC);
  int *flag = reinterpret_cast<int *>(red + 2 * (NT / 32));

  const Unit un = p.units[blockIdx.x];
  const GridDev<T> *gdp = reinterpret_cast<const GridDev<T> *>(p.grids) + un.g;
  SolveState *st = gdp->st;
  LaunchState *ls = p.ls;
  const int kind = p.kind;
  const int tid = threadIdx.x;

  if (p.guard && blockIdx.x == 0 && tid == 0) loop_guard(ls, p);
  if (kind != K2_APPLY && *(volatile int32_t *)&st->done) return;

  const int nx = gdp->nx, ny = gdp->ny, pitch = gdp->pitch, ty = gdp->ty;
  const int i0 = un.sx * TX, j0 = un.sy * ty;
  const int rend = min(j0 + ty, ny);
  const int mlo = j0 - LD, mhi = rend + LD - 1;
  const int rsel = (kind == K2_APPLY) ? 0 : st->rsel;
  const size_t pitch_b = (size_t)pitch * sizeof(T);
  constexpr int SLOTB = G::SLOT * (int)sizeof(T);

  if (tid == 0) {
    for (int s = 0; s < G::NST; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    ctl[0] = 0; ctl[1] = mlo - 1; ctl[2] = mlo - 1;
    for (int w = 0; w < G::NPW; ++w) ctl[3 + w] = mlo - 1;
    fence_mbar_init();
  }
  __syncthreads();

  double acc0 = 0.0, acc1 = 0.0;
  DotAcc<T> dot0, dot1;
  if (tid >= TX) {
    // ---- producer warps
    const int lane = (tid - TX) & 31, pw = (tid - TX) >> 5;
    auto at = [&](const T *plane, int col) { return reinterpret_cast<const char *>(plane + i0 + col); };
    RowCopy c{nullptr, 0, 0, 0};
    if (lane == 0) c = RowCopy{at(gdp->r[rsel], -G::HR), (uint32_t)(G::OFF_R * sizeof(T)), (uint32_t)(G::WR * sizeof(T)), 0};
    else if (lane == 1) { if (kind == K2_ITER) c = RowCopy{at(gdp->q, -G::HR), (uint32_t)(G::OFF_Q * sizeof(T)), (uint32_t)(G::WR * sizeof(T)), 0}; }
    else if (lane - 2 < NZ) c = RowCopy{at(gdp->z[lane - 2], -G::HZ), (uint32_t)((G::OFF_Z + (lane - 2) * G::WZ) * sizeof(T)), (uint32_t)(G::WZ * sizeof(T)), 3};
    else if (lane - 2 == NZ) c = RowCopy{at(gdp->dinv, -G::HZ), (uint32_t)(G::OFF_DI * sizeof(T)), (uint32_t)(G::WZ * sizeof(T)), 3};
    const bool skip_first = (p.dbg_skip_unit == (int)blockIdx.x) && lane == 0 && pw == 0;
    const int last = produce_rows<G::NST>(c, ring_b, SLOTB, full, empty, mlo, mhi, pitch_b, j0, skip_first,
                                          p.timeout_ns, ctl, pw, G::NPW);
    if (lane == 0) ctl[3 + pw] = last;
  } else {
    // ---- compute threads
    const T alpha = (kind == K2_ITER) ? (T)st->alpha : (T)0;
    T *const rout = gdp->r[rsel ^ 1];
    T *const s_out = gdp->s;
    const T *const zwrap = gdp->zwrap;
    // the strips holding the first or last columns apply the periodic side table
    const bool edge = NW > 0 && (i0 < 2 * R + 2 || i0 + TX + 2 * R + 2 > nx);
    int consumed = mlo - 1;
    for (int m = mlo; m <= rend + LD + 1; ++m) {
      bool got = true;
      // r' on row m over [i0-2R, i0+TX+2R)
      if (m <= mhi) {
        const int slot = G::slot(m - mlo);
        got = mbar_wait_bounded(&full[slot], (uint32_t)(((m - mlo) / G::NST) & 1), p.timeout_ns);
        const T *sl = ring + (size_t)slot * G::SLOT;
        T *rnm = rn + (size_t)((m + 8) & (G::NRN - 1)) * G::WRC;
        for (int c = tid; c < G::WRC; c += TX) {
          const int k = c + G::HR - 2 * R;
          T v = sl[G::OFF_R + k];
          if (kind == K2_ITER) v = fma(-alpha, sl[G::OFF_Q + k], v);
          rnm[c] = v;
        }
      }
      // t = D^-1 (Z^T r') on row mt = m - 1 over [i0-R, i0+TX+R)
      const int mt = m - 1;
      if (mt >= j0 && mt <= mhi) {
        const T *sl = ring + (size_t)(G::slot(mt - mlo)) * G::SLOT;
        const T *rnt = rn + (size_t)((mt + 8) & (G::NRN - 1)) * G::WRC;
        T *tm = tt + (size_t)((mt + 8) & (G::NTT - 1)) * G::WTC;
        for (int c = tid; c < G::WTC; c += TX) {
          T acc = (T)0;
          if (mt < ny) {
            const int kz = c + G::HZ - R;
            acc = rnt[c + R];
#pragma unroll
            for (int s = 0; s < NZ; ++s) {
              const T *rrow = rn + (size_t)((mt + P::dy(s) + 8) & (G::NRN - 1)) * G::WRC;
              acc = fma(sl[G::OFF_Z + s * G::WZ + kz], rrow[c + R + P::dx(s)], acc);
            }
            if (edge) {
              const int col = i0 - R + c;
              const int cm = col < 0 ? col + nx : (col >= nx ? col - nx : col);
#pragma unroll
              for (int w = 0; w < (NW > 0 ? NW : 1); ++w)
                if (cm == nx - 1 - P::wcol(w)) acc = fma(zwrap[(size_t)mt * NW + w], rnt[c + R + P::wdx(w)], acc);
            }
            acc *= sl[G::OFF_DI + kz];
          }
          tm[c] = acc;
        }
      }
      // s = Z t on row r = m - 2 - LD
      const int r = m - 2 - LD;
      if (r >= j0 && r < rend) {
        const int col = i0 + tid;
        if (col < nx) {
          const T *tr = tt + (size_t)((r + 8) & (G::NTT - 1)) * G::WTC;
          T acc = tr[tid + R];
#pragma unroll
          for (int s = 0; s < NZ; ++s) {
            const int rowz = r - P::dy(s);           // row of the column holding Z[(col,r), that column]
            const T *slz = ring + (size_t)(G::slot(rowz - mlo)) * G::SLOT;
            const T *trow = tt + (size_t)((rowz + 8) & (G::NTT - 1)) * G::WTC;
            acc = fma(slz[G::OFF_Z + s * G::WZ + tid - P::dx(s) + G::HZ], trow[tid + R - P::dx(s)], acc);
          }
          if (edge) {
#pragma unroll
            for (int w = 0; w < (NW > 0 ? NW : 1); ++w) {
              const int target = P::wdx(w) - 1 - P::wcol(w);   // 0 or 1
              if (col == target) acc = fma(zwrap[(size_t)r * NW + w], tr[tid + R - P::wdx(w)], acc);
            }
          }
          const T *rnr = rn + (size_t)((r + 8) & (G::NRN - 1)) * G::WRC;
          const T rv = rnr[tid + 2 * R];
          const size_t ro = (size_t)r * pitch;
          store_dup(s_out + ro, col, nx, acc);
          if (kind != K2_APPLY) store_dup(rout + ro, col, nx, rv);
          dot0.add(acc, rv);
          dot1.add(rv, rv);
        }
      }
      if (!compute_sync_and<TX>(got)) {
        if (tid == 0) { ctl[0] = 1; flag_timeout(st); }
        break;
      }
      if (m <= mhi) consumed = m;
      // row m-2-LD is finished: its slot may be refilled
      if (tid == 0 && m - 2 - LD >= mlo && m - 2 - LD + G::NST <= mhi) mbar_arrive(&empty[G::slot(m - 2 - LD - mlo)]);
    }
    if (tid == 0) ctl[2] = consumed;
    acc0 = dot0.total();
    acc1 = dot1.total();
  }
  __syncthreads();
  if (tid == 0 && ctl[0]) {
    for (int w = 0; w < G::NPW; ++w)
      for (int m = mlo + w; m <= ctl[3 + w]; m += G::NPW)
        if (m > ctl[2])
          mbar_wait_bounded(&full[G::slot(m - mlo)], (uint32_t)(((m - mlo) / G::NST) & 1), p.timeout_ns);
  }
  if (kind == K2_APPLY) return;
  if (grid_reduce2<NT>(acc0, acc1, gdp->partial, un.u, gdp->n_units, &st->cnt2, red, flag)) {
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

// Mixed precision, refinement step: the binary64 residual r (plane r[rsel] of
// the binary64 grid) scaled by a power of two becomes the binary32 right-hand
// side b of the inner solve.
template <int TX>
__global__ void __launch_bounds__(TX) k_residual_to_f32(const GridDev<double> *g64, const GridDev<float> *g32,
                                                     const Unit *units, double scale) {
  const Unit un = units[blockIdx.x];
  const GridDev<double> &a = g64[un.g];
  const GridDev<float> &f = g32[un.g];
  if (*(volatile int32_t *)&a.st->retired) return;
  const int col = un.sx * TX + threadIdx.x;
  const int j0 = un.sy * a.ty, rend = min(j0 + a.ty, a.ny);
  const double *r = a.r[a.st->rsel];
  const double sc = scale;
  float *b = const_cast<float *>(f.b);
  if (col < a.nx)
    for (int j = j0; j < rend; ++j)
      store_dup(b + (size_t)j * f.pitch, col, a.nx, (float)(r[(size_t)j * a.pitch + col] * sc));
}

// Mixed precision, refinement step: x += e / scale with e the binary32 inner
// solution (x plane of the binary32 grid); the update is done in binary64.
template <int TX>
__global__ void __launch_bounds__(TX) k_correct_f64(const GridDev<double> *g64, const GridDev<float> *g32,
                                                  const Unit *units, double inv_scale) {
  const Unit un = units[blockIdx.x];
  const GridDev<double> &a = g64[un.g];
  const GridDev<float> &f = g32[un.g];
  if (*(volatile int32_t *)&a.st->retired) return;
  const int col = un.sx * TX + threadIdx.x;
  const int j0 = un.sy * a.ty, rend = min(j0 + a.ty, a.ny);
  if (col < a.nx)
    for (int j = j0; j < rend; ++j) {
      double *xr = a.x + (size_t)j * a.pitch;
      store_dup(xr, col, a.nx, fma(to_f64(f.x[(size_t)j * f.pitch + col]), inv_scale, xr[col]));
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
