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
// Group slots of a ring: as many as fit in `budget` bytes, at least live + 1
// and at most 8.
__host__ __device__ constexpr int ring_groups(int budget, int group, int live) {
  return budget / group < live + 1 ? live + 1 : (budget / group > 8 ? 8 : budget / group);
}
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
// binary32 kernels (the inner solves of the mixed mode) take every product
// exactly and sum it with a compensated summation, entirely in the binary32
// pipe: Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM
// J. Sci. Comput. 26, 2005). The product a*b is split into p + e exactly
// (p = fl(a*b), e = fma(a, b, -p)); p is added to the running sum s by
// Knuth's TwoSum, whose exact rounding error joins e in a separate binary32
// error sum c. At the end of a unit the thread's s and c are widened exactly
// and added in binary64, and the units' partials are summed in binary64: the
// result is as accurate as a dot product of the exact products carried in
// twice the binary32 precision, with no binary64 arithmetic per point (the
// FP64 pipe of this GPU is 64 times slower than the FP32 one). The _rn
// intrinsics keep the compiler from contracting or reassociating the steps.
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
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float bv = __fsub_rn(t, s);
    const float z = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    s = t;
    c = __fadd_rn(c, __fadd_rn(z, e));
  }
  __device__ __forceinline__ double total() const { return to_f64(s) + to_f64(c); }
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

// As store_dup, for a thread whose column is fixed: lo = (col < GHOST) and
// hi = (col >= nx - GHOST) are computed once.
template <typename T>
__device__ __forceinline__ void store_col(T *row, int col, int nx, T v, bool lo, bool hi) {
  row[col] = v;
  if (lo)
    for (int c = col + nx; c < nx + GHOST; c += nx) row[c] = v;
  if (hi)
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
  ls->bodies_total += 1;
  const uint64_t now = global_ns();
  if (ls->t0_ns == 0) ls->t0_ns = now;
  const bool late = now - ls->t0_ns > ls->budget_ns;
  if (late) ls->timed_out = 1;
  if (l >= ls->max_launches || late) ls->stop = 1;
  if (l >= ls->max_launches || late || atomicAdd(&ls->active, 0) == 0) clear_loop_condition(ls, p);
}

__device__ __forceinline__ void flag_timeout(SolveState *st) { atomicCAS(&st->status, PCG_OK, PCG_ETIMEOUT); }

// ------------------------------------------------------------ row-group streaming
// A CTA is TX compute threads plus one producer warp, and it is persistent:
// it takes the units blockIdx.x, blockIdx.x + gridDim.x, ... of the launch's
// list (the fixed stride; CTAs are placed round robin on the SMs, so every SM
// gets the same share of equal units, which is what the binary64 kernels,
// bound by each SM's FP64 pipe, need). The claiming instantiations (DYN)
// instead take one unit at a time from a counter in the launch state, so that
// a CTA that finishes early takes more: a batch's units come from grids of
// different sizes that retire at different iterations. Their producer warp
// claims and hands each unit to the compute threads through a small queue in
// shared memory. Which CTA runs a unit does not change its result: partial
// sums are kept per unit and added in unit order.
// The producer streams the input fields of its units, unit after unit
// without a pause, in groups of RB consecutive rows into a ring of NSG group
// slots. Lane f of the producer owns field f and issues one copy per group: a
// 2D tensor tile of RB rows (cp.async.bulk.tensor) when RB > 1, a 1D bulk copy
// of the row (cp.async.bulk) when RB = 1. Lane 0 first arms the slot's "full"
// mbarrier with the group's byte count. The compute threads wait on "full"
// when they reach the first row of a group; once no later step reads the
// group's rows, one of them arrives on the slot's "empty" mbarrier, which the
// producer waits on before it refills the slot. Copies are the unit of cost
// here (each occupies its issuing thread for a few hundred ns on this GPU), so
// several rows per copy is what lets a few CTAs per SM keep HBM busy.

// control words at the start of shared memory (after the barriers); the
// claiming kernels' unit queue (UQ entries) fills the rest of the 64 bytes
enum { CTL_ABORT = 0, CTL_ARMED = 1, CTL_SEEN = 2, CTL_FLAG = 3, CTL_PUB = 4, CTL_CONS = 5, CTL_CUR = 6, CTL_QUEUE = 8 };
constexpr int UQ = 8;

struct FieldCopy {
  const char *src;      // RB = 1: element (first box column, row 0) of the plane, as bytes
  const void *tmap;     // RB > 1: tensor map of the plane with this field's box
  int64_t pitch_b;      // RB = 1: bytes between rows of the plane
  int32_t x;            // RB > 1: first box column, counted from the plane's first stored column
  uint32_t dst;         // byte offset of the field in a group slot
  uint32_t bytes;       // bytes of the field in one group
};

// 2D tensor tile (box of the map) at column x, row y of the map into shared
// memory (128-byte aligned); completion counted on bar. x * sizeof(element)
// is a multiple of 16 by construction of every caller.
__device__ __forceinline__ void tma_2d_g2s(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// The tensor maps live in global memory, written by the host: acquire them
// for the tensor-map proxy before the first copy that uses them.
__device__ __forceinline__ void tensormap_acquire(const void *tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

// Wait for a phase of an mbarrier, giving up after timeout_ns or as soon as
// the CTA's abort word is set.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, uint64_t timeout_ns,
                                                   const volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0 && (*abort || global_ns() - t0 > timeout_ns)) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// mbar_arrive in the thread where `on` holds, as one predicated instruction
// (no branch around it)
__device__ __forceinline__ void mbar_arrive_if(uint64_t *bar, bool on) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n @p mbarrier.arrive.shared::cta.b64 _, [%0];\n}\n" ::"r"(
          smem_addr(bar)),
      "r"((uint32_t)on)
      : "memory");
}

// Barrier of the NC compute threads only (named barrier 1), with an AND vote.
template <int NC>
__device__ __forceinline__ bool compute_sync_and(bool v) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n barrier.cta.red.and.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(NC)
      : "memory");
  return out != 0;
}
template <int NC>
__device__ __forceinline__ void compute_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
}

// A CTA's next unit after unit ui when ui's whole grid is to be skipped
// (done): the first index at or past u_end = u_off + n_units of that grid in
// the CTA's stride. Units of a grid are contiguous in a launch's list.
__device__ __forceinline__ int skip_grid(int ui, int u_end) {
  const int g = (int)gridDim.x;
  return u_end <= ui ? ui + g : ui + (u_end - ui + g - 1) / g * g;
}

// Wait until pred() holds, giving up after timeout_ns (one thread).
template <class Pred>
__device__ __forceinline__ bool spin_bounded(Pred pred, uint64_t timeout_ns) {
  if (pred()) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (pred()) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > timeout_ns) return false;
  }
}

// Claiming: the launch's next unit (lane 0 takes it, the warp shares it).
__device__ __forceinline__ int claim_unit(const KParams &p, int lane) {
  int ui = 0;
  if (lane == 0) ui = (int)atomicAdd(&p.ls->claim_next, 1u);
  return __shfl_sync(0xffffffffu, ui, 0);
}

// Claiming: append unit v (-1: no more) to the unit queue once there is room,
// as the producer's pub-th entry. False if the compute threads took no entry
// for timeout_ns (the CTA is then marked aborting).
__device__ __forceinline__ bool queue_push(volatile int *ctl, int pub, int v, int lane, uint64_t timeout_ns) {
  bool ok = true;
  if (lane == 0) {
    ok = spin_bounded([&] { return pub - ctl[CTL_CONS] < UQ; }, timeout_ns);
    if (ok) {
      ctl[CTL_QUEUE + pub % UQ] = v;
      __threadfence_block();
      ctl[CTL_PUB] = pub + 1;
    } else {
      ctl[CTL_ABORT] = 1;
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0);
}

// The producer warp's loop: lane f issues the copies of field f of every
// group of the CTA's units, in order. setup(ui, f, c, has, mlo, ng, u_end)
// describes unit ui's field f (returns false when ui's grid is to be skipped,
// with u_end the end of that grid's units). Returns the number of groups
// armed. With the fixed stride the compute threads walk the same units and
// take the same skip decisions themselves, and the producer stops early once
// the CTA is aborting. With DYN a skipped grid's remaining units are passed
// over by raising the claim counter past them, every other unit is queued for
// the compute threads before its copies are issued, units are still queued
// (without copies) once the CTA is aborting, so that the compute threads join
// every unit's reduction, and -1 ends the queue.
template <int NSG, int RB, bool DYN, class Setup>
__device__ __forceinline__ uint32_t produce_all(const KParams &p, unsigned char *ring, int group_bytes, uint64_t *full,
                                                uint64_t *empty, volatile int *ctl, Setup setup) {
  const int lane = threadIdx.x & 31;
  uint32_t gq = 0;
  int last_g = -1;
  int pub = 0;             // DYN: units queued
  bool stopped = false;    // DYN: no more copies, the CTA is aborting
  for (int ui = DYN ? claim_unit(p, lane) : (int)blockIdx.x; ui < p.n_units;
       ui = DYN ? claim_unit(p, lane) : ui + (int)gridDim.x) {
    FieldCopy c{};
    bool has = false;
    int mlo = 0, ng = 0, u_end = 0;
    if constexpr (DYN) {
      if (!__shfl_sync(0xffffffffu, setup(ui, lane, c, has, mlo, ng, u_end), 0)) {
        if (lane == 0 && u_end > ui + 1) atomicMax(&p.ls->claim_next, (unsigned)u_end);
        continue;
      }
      if (!queue_push(ctl, pub++, ui, lane, p.timeout_ns)) return gq;
      if (stopped) continue;
    } else if (!setup(ui, lane, c, has, mlo, ng, u_end)) {
      ui = skip_grid(ui, u_end) - (int)gridDim.x;
      continue;
    }
    const int g_un = p.units[ui].g;
    const bool skip_first = (p.dbg_skip_unit == ui) && lane == 0;
    if constexpr (RB > 1)
      if (has && g_un != last_g) tensormap_acquire(c.tmap);
    last_g = g_un;
    const uint32_t total = __reduce_add_sync(0xffffffffu, has ? c.bytes : 0u);
    for (int q = 0; q < ng; ++q, ++gq) {
      const uint32_t slot = gq % NSG, fill = gq / NSG;
      if (fill > 0) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait_or_abort(&empty[slot], (fill - 1) & 1u, p.timeout_ns, &ctl[CTL_ABORT]);
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          if (lane == 0) ctl[CTL_ABORT] = 1;
          if constexpr (!DYN) return gq;
          stopped = true;
          break;
        }
      }
      if (lane == 0) mbar_arrive_expect_tx(&full[slot], total);
      __syncwarp();
      if (has && !(skip_first && q == 0)) {
        fence_proxy_async();
        unsigned char *dst = ring + (size_t)slot * group_bytes + c.dst;
        const int m0 = mlo + q * RB;
        if constexpr (RB == 1) bulk_g2s(dst, c.src + (ptrdiff_t)m0 * c.pitch_b, c.bytes, &full[slot]);
        else tma_2d_g2s(dst, c.tmap, c.x, m0 + GY, &full[slot]);
      }
    }
  }
  if constexpr (DYN) queue_push(ctl, pub, -1, lane, p.timeout_ns);
  return gq;
}

// The compute threads' first unit (k = 0) and the ones after unit ui (k-th):
// the fixed stride, or with DYN the producer's k-th queue entry, which thread
// 0 waits for (bounded) and shares through ctl[CTL_CUR]. -1: no more units.
template <bool DYN, int NC>
__device__ __forceinline__ int compute_unit(const KParams &p, volatile int *ctl, int k, int ui) {
  if constexpr (!DYN) {
    ui = k == 0 ? (int)blockIdx.x : ui + (int)gridDim.x;
    return ui < p.n_units ? ui : -1;
  } else {
    if (threadIdx.x == 0) {
      const bool ok = spin_bounded([&] { return ctl[CTL_PUB] > k; }, p.timeout_ns);
      __threadfence_block();
      ctl[CTL_CUR] = ok ? ctl[CTL_QUEUE + k % UQ] : -1;
      if (!ok) ctl[CTL_ABORT] = 1;
    }
    compute_sync<NC>();
    ui = ctl[CTL_CUR];
    compute_sync<NC>();
    if (threadIdx.x == 0) ctl[CTL_CONS] = k + 1;
    return ui;
  }
}

// End of a claiming launch: the last CTA to leave resets the claim counters
// for the next launch (every CTA has finished claiming by then).
__device__ __forceinline__ void launch_exit(LaunchState *ls) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ls->claim_exit, 1u) + 1u == gridDim.x) {
      ls->claim_next = 0u;
      ls->claim_exit = 0u;
      __threadfence();
    }
  }
}

// Shared-memory geometry common to both kernels: barriers and control words
// in the first 256 bytes of a 128-byte aligned base, then the group ring.
template <int NSG>
struct RingCtl {
  static_assert(NSG <= 12, "barrier area");
  uint64_t *full, *empty;
  volatile int *ctl;
  unsigned char *ring;
  __device__ __forceinline__ explicit RingCtl(unsigned char *base) {
    full = reinterpret_cast<uint64_t *>(base);
    empty = full + NSG;
    ctl = reinterpret_cast<volatile int *>(base + 192);
    ring = base + 256;
  }
};

__device__ __forceinline__ unsigned char *align128(unsigned char *p) {
  const uint32_t a = smem_addr(p);
  return p + ((128u - (a & 127u)) & 127u);
}

// Sum (a, b) over the NC compute threads; the totals end in thread 0.
template <int NC>
__device__ __forceinline__ void compute_sum2(double &a, double &b, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  compute_sync<NC>();
  if (lane == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
  compute_sync<NC>();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int i = 0; i < NC / 32; ++i) { sa += red[2 * i]; sb += red[2 * i + 1]; }
    a = sa; b = sb;
  }
}

// Write one unit's partials; return true (in every compute thread) if it was
// the last unit of its grid to arrive, in which case (sa, sb) hold the grid's
// totals in thread 0, summed in unit order.
template <int NC>
__device__ __forceinline__ bool unit_reduce2(double &sa, double &sb, double *partial, int u, int n_units,
                                             uint32_t *counter, double *red, volatile int *flag) {
  compute_sum2<NC>(sa, sb, red);
  if (threadIdx.x == 0) {
    partial[2 * u] = sa;
    partial[2 * u + 1] = sb;
    __threadfence();
    const uint32_t prev = atomicAdd(counter, 1u);
    *flag = (prev == (uint32_t)(n_units - 1));
  }
  compute_sync<NC>();
  if (!*flag) return false;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < n_units; t += NC) {
    a += __ldcg(partial + 2 * t);
    b += __ldcg(partial + 2 * t + 1);
  }
  compute_sum2<NC>(a, b, red);
  if (threadIdx.x == 0) {
    sa = a; sb = b;
    atomicExch(counter, 0u);
  }
  return true;
}

// Drain at the end of a CTA that aborted: wait (bounded) for the groups armed
// but never seen by the compute threads, so no copy lands after exit.
template <int NSG>
__device__ __forceinline__ void drain_groups(const RingCtl<NSG> &rc, uint64_t timeout_ns) {
  if (threadIdx.x == 0 && rc.ctl[CTL_ABORT]) {
    const uint32_t armed = (uint32_t)rc.ctl[CTL_ARMED];
    for (uint32_t g = (uint32_t)rc.ctl[CTL_SEEN]; g < armed; ++g)
      mbar_wait_bounded(&rc.full[g % NSG], (g / NSG) & 1u, timeout_ns);
  }
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
  static constexpr int WDN = TX + 2;                 // d' ring: [i0-1, i0+TX+1)
  static constexpr int NDN = 4;                      // rows of d' kept (a power of two)
  static constexpr int RB = sizeof(T) == 4 ? 4 : 1;  // rows per group
  static constexpr int FA = RB > 1 ? 128 : 16;       // alignment of a field in a group
  __host__ __device__ static constexpr int fb(int w) { return round_up_c(RB * w * (int)sizeof(T), FA); }
  static constexpr int OFF_S = 0, OFF_D = OFF_S + fb(WS), OFF_N = OFF_D + fb(WS), OFF_E = OFF_N + fb(WT),
                       OFF_A = OFF_E + fb(WE), OFF_X = OFF_A + fb(WT), GROUP = OFF_X + fb(WT);   // bytes
  // group slots: the groups a step reads (rows m-3..m) plus at least one in
  // flight. The binary32 kernel is bound by its compute warps, so its ring is
  // kept small (about 40 KB) for CTAs per SM. binary64: 8 rows (4 in flight);
  // strips wider than 64 columns keep 5 (1 in flight), which lets 6 CTAs
  // instead of 4 share an SM (measured faster on 124-column strips).
  static constexpr int LIVE = (3 + RB - 1) / RB + 1;
  static constexpr int NSG = RB == 1 ? (TX > 64 ? 5 : 8) : ring_groups(40000, GROUP, LIVE);
  // NGRP warp groups of TX compute threads (with 2, each step's work is split:
  // group 0 d', the x update and the waits, group 1 q = A d' and its stores;
  // measured no faster than 1 on this GPU), then the producer warp
  // NCG: compute threads of a group, the strip width rounded up to whole
  // warps (a strip of 64 - 2R columns lets the t phase of the preconditioner
  // kernel cover its TX + 2R columns with whole warps, no extra pass)
  static constexpr int NCG = round_up_c(TX, 32);
  static constexpr int NGRP = 1, NC = NGRP * NCG, NT = NC + 32;
  static constexpr size_t SMEM = 128 + 256 + (size_t)NSG * GROUP + sizeof(T) * (size_t)NDN * WDN + 16 * (NT / 32) + 64;
};

// Compile-time row bookkeeping of the unrolled step loops: floor division
// and non-negative remainder.
__host__ __device__ constexpr int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__host__ __device__ constexpr int pmod(int a, int b) { return ((a % b) + b) % b; }

// A compute thread's column store with its periodic copies. Device grids are
// at least GHOST columns wide (setup refuses narrower ones), so a column has at
// most two copies, col + nx (if col < GHOST) and col - nx (if col >= nx -
// GHOST). A thread past the strip or the grid (ok = false) stores nothing:
// three predicated stores, no branch.
template <typename T>
struct ColStore {
  int col, da, db;
  bool own, pa, pb;
  __device__ __forceinline__ void init(int c, int n, bool ok) {
    col = c; own = ok;
    pa = ok && c < GHOST; da = c + n;
    pb = ok && c >= n - GHOST; db = c - n;
  }
  __device__ __forceinline__ void put(T *row, T v) const {
    if (own) row[col] = v;
    if (pa) row[da] = v;
    if (pb) row[db] = v;
  }
};

// One unit of k_stencil on the compute side. The step loop is unrolled by 8
// (a multiple of RB and of the d' ring), so the row-in-group, the ring rows
// and which group holds a row are compile-time; only the group slot bases
// (gb[0] for the group of row m, gb[1] the one before, ...) are registers.
template <typename T, int TX, int KIND>
struct K1Unit {
  using G = K1Geom<T, TX>;
  static constexpr int kind = KIND;
  static constexpr int RB = G::RB, NSG = G::NSG, ESZ = (int)sizeof(T);
  static constexpr int WIN = 4;                              // rows m-3 .. m are read by a step
  static constexpr int NGB = (WIN - 1 + RB - 1) / RB + 1;    // groups those rows can span
  static_assert(8 % RB == 0 && 8 % G::NDN == 0, "unroll by 8");
  __device__ static constexpr int gback(int K, int k) { return fdiv(K, RB) - fdiv(K - k, RB); }

  const unsigned char *ring_lo, *ring_hi;   // ring bounds (+ this thread's column)
  const unsigned char *gb[NGB];
  const unsigned char *next_sb;
  T *dn;                                    // d' ring (+ this thread's column)
  uint64_t *full, *empty;
  const volatile int *abort;
  T *d_out, *x_out, *q_out, *r_out;
  uint64_t timeout_ns;
  uint32_t fslot, fpar, eslot;
  int tid, lt, grp, mlo, nr1, nrows, pitch, ng, nseen, nrel;   // lt: column in the strip, grp: warp group
  bool col_ok;
  ColStore<T> cs;
  T beta, pend;
  DotAcc<T> dot0, dot1;

  __device__ __forceinline__ void begin(const unsigned char *ring, uint32_t gbase) {
    ring_lo = ring + lt * ESZ;
    ring_hi = ring_lo + (size_t)NSG * G::GROUP;
    fslot = gbase % NSG;
    fpar = (gbase / NSG) & 1u;
    eslot = fslot;
    next_sb = ring_lo + (size_t)fslot * G::GROUP;
#pragma unroll
    for (int j = 0; j < NGB; ++j) gb[j] = next_sb;
    nseen = 0;
    nrel = 0;
  }
  template <int F>
  __device__ __forceinline__ static const T *fld(const unsigned char *sb, int irow, int w) {
    return reinterpret_cast<const T *>(sb + F) + irow * w;
  }

  // CHK = false: a step of the unit's steady part, where every phase is
  // active (the range checks are skipped).
  template <int K, bool CHK>
  __device__ __forceinline__ bool step(int rel) {
    constexpr int I = K % RB;
    if constexpr (I == 0) {
#pragma unroll
      for (int j = NGB - 1; j > 0; --j) gb[j] = gb[j - 1];
      gb[0] = next_sb;
      next_sb += G::GROUP;
      if (next_sb == ring_hi) next_sb = ring_lo;
    }
    const bool ga = G::NGRP == 1 || grp == 0, gb1 = G::NGRP == 1 || grp == 1;
    // Loads of a step come before its shared-memory stores: q on row m - 2
    // first (it reads d' rows written in earlier steps), then d' on row m.
    // q = A d' on row r = m - 2 (rel - 3 = r - j0)
    // every thread computes (the threads past the strip or the grid read
    // in-bounds shared memory and store nothing; their dot terms are zero)
    const bool qrow = !CHK || (rel >= 3 && rel - 3 < nrows);
    if (gb1 && qrow) {
      const unsigned char *br = gb[gback(K, 2)], *bs = gb[gback(K, 3)];
      constexpr int IR = pmod(K - 2, RB), IS = pmod(K - 3, RB);
      const T *dr = dn + pmod(K - 2, G::NDN) * G::WDN;
      const T *ds = dn + pmod(K - 3, G::NDN) * G::WDN;
      const T *dnn = dn + pmod(K - 1, G::NDN) * G::WDN;
      const T *Nr = fld<G::OFF_N>(br, IR, G::WT), *Ns = fld<G::OFF_N>(bs, IS, G::WT);
      const T *Er = fld<G::OFF_E>(br, IR, G::WE), *Ar = fld<G::OFF_A>(br, IR, G::WT);
      const T *Xr = fld<G::OFF_X>(br, IR, G::WT), *Dr = fld<G::OFF_D>(br, IR, G::WS);
      const T c_ctr = dr[1];
      T av = -Ns[0] * ds[1];
      av = fma(-Er[G::H - 1], dr[0], av);
      av = fma(Ar[0], c_ctr, av);
      av = fma(-Er[G::H], dr[2], av);
      av = fma(-Nr[0], dnn[1], av);
      const size_t ro = (size_t)(mlo + rel - 2) * pitch;
      if (kind == K1_ITER) {
        cs.put(d_out + ro, c_ctr);
        if constexpr (G::NGRP == 1) cs.put(x_out + ro, fma(pend, Dr[G::H], Xr[0]));
        cs.put(q_out + ro, av);
        dot0.add(col_ok ? c_ctr : (T)0, col_ok ? av : (T)0);
      } else if (kind == K1_SPMV) {
        cs.put(q_out + ro, av);
      } else {
        const T bv = col_ok ? Xr[0] : (T)0;
        const T rv = col_ok ? bv - av : (T)0;
        cs.put(r_out + ro, rv);
        dot0.add(rv, rv);
        dot1.add(bv, bv);
      }
    }
    if constexpr (G::NGRP == 2 && KIND == K1_ITER) {
      // x += pending d_old on row r (group 0)
      if (grp == 0 && qrow && col_ok) {
        const unsigned char *br = gb[gback(K, 2)];
        constexpr int IR = pmod(K - 2, RB);
        const T *Xr = fld<G::OFF_X>(br, IR, G::WT), *Dr = fld<G::OFF_D>(br, IR, G::WS);
        cs.put(x_out + (size_t)(mlo + rel - 2) * pitch, fma(pend, Dr[G::H], Xr[0]));
      }
    }
    // last: d' on row m (the only part that waits for streamed data)
    bool got = true, waited = false;
    if (ga && (!CHK || rel <= nr1)) {                  // row m = mlo + rel is streamed
      if constexpr (I == 0) {
        got = mbar_wait_or_abort(&full[fslot], fpar, timeout_ns, abort);
        waited = true;
        if (++fslot == (uint32_t)NSG) { fslot = 0; fpar ^= 1u; }
      }
      const T *S = fld<G::OFF_S>(gb[0], I, G::WS), *D = fld<G::OFF_D>(gb[0], I, G::WS);
      T *dnm = dn + (K & (G::NDN - 1)) * G::WDN;
      // d' on row m over columns [i0-1, i0+TX+1) (threads past the row's width idle)
      if (G::NCG <= G::WDN || lt < G::WDN) {
        T v = S[G::H - 1];
        if (kind == K1_ITER) v = fma(beta, D[G::H - 1], v);
        dnm[0] = v;
      }
      if (lt < G::WDN - G::NCG) {                     // columns past the group's threads
        T v2 = S[G::H - 1 + G::NCG];
        if (kind == K1_ITER) v2 = fma(beta, D[G::H - 1 + G::NCG], v2);
        dnm[G::NCG] = v2;
      }
    }
    if constexpr (I == 0) {
      if (!compute_sync_and<G::NC>(got)) return false;
    } else {
      compute_sync<G::NC>();
    }
    if (waited) ++nseen;
    // row m - 3 is finished: at the last row of its group, release the group
    if constexpr (pmod(K - 2, RB) == 0) {
      if (!CHK || rel >= 3) {
        mbar_arrive_if(&empty[eslot], tid == 0);
        if (++eslot == (uint32_t)NSG) eslot = 0;
        ++nrel;
      }
    }
    return true;
  }

  // All steps of the unit (rel = 0 .. nrows + 2); releases the unit's groups.
  // Blocks of 8 steps inside [3, nr1] (both phases active) skip the checks.
  __device__ __forceinline__ bool run() {
    const int last = nrows + 2;
    for (int b = 0; b <= last; b += 8) {
      if (b >= 3 && b + 7 <= nr1) {
#define PCG_K1_STEADY(K) \
  if (!step<K, false>(b + K)) return false;
        PCG_K1_STEADY(0) PCG_K1_STEADY(1) PCG_K1_STEADY(2) PCG_K1_STEADY(3)
        PCG_K1_STEADY(4) PCG_K1_STEADY(5) PCG_K1_STEADY(6) PCG_K1_STEADY(7)
#undef PCG_K1_STEADY
        continue;
      }
#define PCG_K1_STEP(K) \
  if (b + K > last) break; \
  if (!step<K, true>(b + K)) return false;
      PCG_K1_STEP(0) PCG_K1_STEP(1) PCG_K1_STEP(2) PCG_K1_STEP(3)
      PCG_K1_STEP(4) PCG_K1_STEP(5) PCG_K1_STEP(6) PCG_K1_STEP(7)
#undef PCG_K1_STEP
    }
    for (; nrel < ng; ++nrel) {
      mbar_arrive_if(&empty[eslot], tid == 0);
      if (++eslot == (uint32_t)NSG) eslot = 0;
    }
    return true;
  }
};

template <typename T, int TX, int KIND, bool DYN>
__global__ void __launch_bounds__(K1Geom<T, TX>::NT) k_stencil(KParams p) {
  using G = K1Geom<T, TX>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align128(smem_raw);
  const RingCtl<G::NSG> rc(base);
  T *dn = reinterpret_cast<T *>(rc.ring + (size_t)G::NSG * G::GROUP);
  double *red = reinterpret_cast<double *>(dn + (size_t)G::NDN * G::WDN);
  constexpr int kind = KIND;
  const int tid = threadIdx.x;
  LaunchState *ls = p.ls;

  if (tid == 0) {
    for (int s = 0; s < G::NSG; ++s) { mbar_init(&rc.full[s], 1); mbar_init(&rc.empty[s], 1); }
    rc.ctl[CTL_ABORT] = 0; rc.ctl[CTL_ARMED] = 0; rc.ctl[CTL_SEEN] = 0; rc.ctl[CTL_FLAG] = 0;
    rc.ctl[CTL_PUB] = 0; rc.ctl[CTL_CONS] = 0;
    fence_mbar_init();
  }
  __syncthreads();

  auto skip_unit = [&](const SolveState *st) {
    if (kind == K1_ITER || kind == K1_RESID_INIT) return *(const volatile int32_t *)&st->done != 0;
    if (kind == K1_RESID_CHECK) return *(const volatile int32_t *)&st->retired != 0;
    return false;
  };

  if (tid >= G::NC) {
    // ---- producer warp
    auto setup = [&](int ui, int f, FieldCopy &c, bool &has, int &mlo, int &ng, int &u_end) -> bool {
      const Unit un = p.units[ui];
      const GridDev<T> *gdp = reinterpret_cast<const GridDev<T> *>(p.grids) + un.g;
      u_end = gdp->u_off + gdp->n_units;
      if (skip_unit(gdp->st)) return false;
      const int i0 = un.sx * TX, j0 = gdp->own0 + un.sy * gdp->ty;
      const int mhi = min(j0 + gdp->ty, gdp->own1);
      mlo = j0 - 1;
      ng = (mhi - mlo + G::RB) / G::RB;
      const int dsel = gdp->st->dsel;
      const T *src_s = (kind == K1_ITER) ? gdp->s : (kind == K1_SPMV) ? gdp->d[0] : gdp->x;
      const int tm_s = (kind == K1_ITER) ? TM_WS_S : (kind == K1_SPMV) ? TM_WS_D0 : TM_WS_X;
      const TensorMapBytes *tm = gdp->tm;
      auto mk = [&](const T *plane, int tmi, int col, int off, int w) {
        c.src = reinterpret_cast<const char *>(plane + i0 + col);
        c.tmap = tm ? (const void *)(tm + tmi) : nullptr;
        c.pitch_b = (int64_t)gdp->pitch * (int64_t)sizeof(T);
        c.x = 128 / (int)sizeof(T) + i0 + col;
        c.dst = (uint32_t)off;
        c.bytes = (uint32_t)(G::RB * w * (int)sizeof(T));
      };
      has = true;
      switch (f) {
        case 0: mk(src_s, tm_s, -G::H, G::OFF_S, G::WS); break;
        case 1: mk(gdp->d[dsel], dsel ? TM_WS_D1 : TM_WS_D0, -G::H, G::OFF_D, G::WS); has = kind == K1_ITER; break;
        case 2: mk(gdp->cn, TM_WT_CN, 0, G::OFF_N, G::WT); break;
        case 3: mk(gdp->ce, TM_WE_CE, -G::H, G::OFF_E, G::WE); break;
        case 4: mk(gdp->a, TM_WT_A, 0, G::OFF_A, G::WT); break;
        case 5: mk(kind == K1_ITER ? gdp->x : gdp->b, kind == K1_ITER ? TM_WT_X : TM_WT_B, 0, G::OFF_X, G::WT);
                has = kind != K1_SPMV; break;
        default: has = false; break;
      }
      return true;
    };
    const uint32_t gq =
        produce_all<G::NSG, G::RB, DYN>(p, rc.ring, G::GROUP, rc.full, rc.empty, rc.ctl, setup);
    if (tid == G::NC) rc.ctl[CTL_ARMED] = (int)gq;
  } else {
    // ---- compute threads
    uint32_t gbase = 0, seen = 0;
    bool aborted = false;
    for (int k = 0, ui = compute_unit<DYN, G::NC>(p, rc.ctl, 0, 0); ui >= 0;
         ui = compute_unit<DYN, G::NC>(p, rc.ctl, ++k, ui)) {
      const Unit un = p.units[ui];
      const GridDev<T> *gdp = reinterpret_cast<const GridDev<T> *>(p.grids) + un.g;
      SolveState *st = gdp->st;
      if constexpr (!DYN) {                  // (claimed units of skipped grids are never queued)
        if (skip_unit(st)) {
          ui = skip_grid(ui, gdp->u_off + gdp->n_units) - (int)gridDim.x;
          continue;
        }
      }
      const int nx = gdp->nx, ny = gdp->ny;
      const int i0 = un.sx * TX, j0 = gdp->own0 + un.sy * gdp->ty;
      const int rend = min(j0 + gdp->ty, gdp->own1);
      const int mlo = j0 - 1, mhi = rend;
      const int ng = (mhi - mlo + G::RB) / G::RB;
      double acc0 = 0.0, acc1 = 0.0;
      if (!aborted) {
        K1Unit<T, TX, KIND> cx;
        cx.tid = tid; cx.grp = tid / G::NCG; cx.lt = tid - cx.grp * G::NCG;
        cx.dn = dn + cx.lt; cx.full = rc.full; cx.empty = rc.empty; cx.abort = &rc.ctl[CTL_ABORT];
        cx.timeout_ns = p.timeout_ns;
        cx.begin(rc.ring, gbase);
        cx.mlo = mlo; cx.nr1 = mhi - mlo; cx.nrows = rend - j0; cx.ng = ng;
        cx.pitch = gdp->pitch;
        cx.col_ok = cx.lt < TX && i0 + cx.lt < nx;
        cx.cs.init(i0 + cx.lt, nx, cx.col_ok);
        cx.beta = (kind == K1_ITER) ? (T)st->beta : (T)0;
        cx.pend = (kind == K1_ITER) ? (T)st->pending : (T)0;
        const int dsel = st->dsel;
        cx.d_out = gdp->d[dsel ^ 1]; cx.x_out = gdp->x; cx.q_out = gdp->q; cx.r_out = gdp->r[st->rsel];
        if (!cx.run()) aborted = true;
        seen = gbase + (uint32_t)cx.nseen;
        acc0 = cx.dot0.total();
        acc1 = cx.dot1.total();
      }
      gbase += ng;
      if (aborted && tid == 0) { rc.ctl[CTL_ABORT] = 1; flag_timeout(st); }
      if (kind == K1_SPMV) continue;
      if (unit_reduce2<G::NC>(acc0, acc1, gdp->partial, un.u, gdp->n_units, &st->cnt1, red, &rc.ctl[CTL_FLAG])) {
        if (tid == 0) {
          if (kind == K1_ITER) {
            const double dq = acc0;
            st->dq = dq;
            st->pending = 0.0;
            st->dsel = st->dsel ^ 1;
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
    if (tid == 0) rc.ctl[CTL_SEEN] = (int)seen;
  }
  __syncthreads();
  drain_groups<G::NSG>(rc, p.timeout_ns);
  if constexpr (DYN) launch_exit(ls);
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
  static constexpr int RB = sizeof(T) == 4 ? 2 : 1;  // rows per group
  static constexpr int FA = RB > 1 ? 128 : 16;
  __host__ __device__ static constexpr int fb(int w) { return round_up_c(RB * w * (int)sizeof(T), FA); }
  static constexpr int OFF_R = 0, OFF_Q = fb(WR), OFF_Z = 2 * fb(WR), OFF_DI = OFF_Z + NZ * fb(WZ),
                       GROUP = OFF_DI + fb(WZ);      // bytes
  // group slots: the groups a step reads (rows m-2-LD..m) plus at least one
  // in flight. Both precisions are bound by their compute warps, so shared
  // memory goes to CTAs per SM: binary64 keeps one row ahead, binary32 about
  // 42 KB of ring.
  static constexpr int LIVE = (LD + 2 + RB - 1) / RB + 1;
  static constexpr int NSG = RB == 1 ? LD + 4 : ring_groups(42000, GROUP, LIVE);
  // NGRP warp groups of TX compute threads (with 2, each step's work is split:
  // group 0 t, r' and the waits, group 1 s = Z t and its stores; measured no
  // faster than 1 on this GPU), then the producer warp
  static constexpr int NCG = round_up_c(TX, 32);      // compute threads of a group (whole warps)
  static constexpr int NGRP = 1, NC = NGRP * NCG, NT = NC + 32;
  static constexpr size_t SMEM = 128 + 256 + (size_t)NSG * GROUP +
                                 sizeof(T) * ((size_t)NRN * WRC + (size_t)NTT * WTC) + 16 * (NT / 32) + 64;
  // binary64 strips wider than 64 columns whose ring lets 6 CTAs share an SM
  // (tril(A) at 124 columns): registers for those 6
  static constexpr int MINB = (sizeof(T) == 8 && TX > 64 && 6 * (SMEM + 1024) <= 233472) ? 6 : 1;
};

// One unit of k_precond on the compute side, unrolled by 8 steps like K1Unit.
template <typename T, int TX, class P, int KIND>
struct K2Unit {
  using G = K2Geom<T, TX, P>;
  static constexpr int kind = KIND;
  static constexpr int R = P::R, LD = P::LD, NZ = P::NZ, NW = P::NW;
  static constexpr int RB = G::RB, NSG = G::NSG, ESZ = (int)sizeof(T);
  static constexpr int WIN = LD + 3;                         // rows m-2-LD .. m are read by a step
  static constexpr int NGB = (WIN - 1 + RB - 1) / RB + 1;
  static constexpr int FBZ = G::fb(G::WZ);
  static_assert(8 % RB == 0 && 8 % G::NRN == 0 && 8 % G::NTT == 0, "unroll by 8");
  __device__ static constexpr int gback(int K, int k) { return fdiv(K, RB) - fdiv(K - k, RB); }

  const unsigned char *ring_lo, *ring_hi;
  const unsigned char *gb[NGB];
  const unsigned char *next_sb;
  T *rn, *tt;                              // rings (+ this thread's column)
  uint64_t *full, *empty;
  const volatile int *abort;
  T *rout, *s_out;
  const T *zwrap;
  uint64_t timeout_ns;
  uint32_t fslot, fpar, eslot;
  int tid, lt, grp, nx, ny, mlo, j0, i0, nr1, nrows, pitch, ng, nseen, nrel, col;
  bool col_ok, edge;
  ColStore<T> cs;
  T alpha;
  DotAcc<T> dot0, dot1;

  __device__ __forceinline__ void begin(const unsigned char *ring, uint32_t gbase) {
    ring_lo = ring + lt * ESZ;
    ring_hi = ring_lo + (size_t)NSG * G::GROUP;
    fslot = gbase % NSG;
    fpar = (gbase / NSG) & 1u;
    eslot = fslot;
    next_sb = ring_lo + (size_t)fslot * G::GROUP;
#pragma unroll
    for (int j = 0; j < NGB; ++j) gb[j] = next_sb;
    nseen = 0;
    nrel = 0;
  }
  __device__ __forceinline__ static const T *fld(const unsigned char *sb, int off, int irow, int w) {
    return reinterpret_cast<const T *>(sb + off) + irow * w;
  }

  // t = D^-1 (Z^T r') on row mt (phase KT = K - 1) at column c = lt + dc of
  // [i0-R, i0+TX+R): dc = 0 (main) or TX (the right halo columns)
  template <int KT>
  __device__ __forceinline__ T tcol(const unsigned char *bz, int dc, int mt) const {
    constexpr int IZ = pmod(KT, RB);
    const T *rnt = rn + pmod(KT, G::NRN) * G::WRC + dc;
    T acc = rnt[R];
#pragma unroll
    for (int s = 0; s < NZ; ++s) {
      const T *rrow = rn + pmod(KT + P::dy(s), G::NRN) * G::WRC + dc;
      acc = fma(fld(bz, G::OFF_Z + s * FBZ, IZ, G::WZ)[G::HZ - R + dc], rrow[R + P::dx(s)], acc);
    }
    if (edge && mt < ny) {                   // rows >= ny: zero t (Z, D^-1 and r' are zero there)
      const int cg = i0 - R + lt + dc;
      const int cm = cg < 0 ? cg + nx : (cg >= nx ? cg - nx : cg);
#pragma unroll
      for (int w = 0; w < (NW > 0 ? NW : 1); ++w)
        if (cm == nx - 1 - P::wcol(w)) acc = fma(zwrap[(size_t)mt * NW + w], rnt[R + P::wdx(w)], acc);
    }
    return acc * fld(bz, G::OFF_DI, IZ, G::WZ)[G::HZ - R + dc];
  }

  // CHK = false: a step of the unit's steady part, where every phase is
  // active (the range checks are skipped).
  template <int K, bool CHK>
  __device__ __forceinline__ bool step(int rel) {
    constexpr int I = K % RB;
    if constexpr (I == 0) {
#pragma unroll
      for (int j = NGB - 1; j > 0; --j) gb[j] = gb[j - 1];
      gb[0] = next_sb;
      next_sb += G::GROUP;
      if (next_sb == ring_hi) next_sb = ring_lo;
    }
    // Loads of a step come before its shared-memory stores: s on row
    // m - 2 - LD (reads t rows of earlier steps), t on row m - 1 (reads r'
    // rows of earlier steps), then r' on row m, the only part that waits for
    // streamed data.
    const bool ga = G::NGRP == 1 || grp == 0, gb1 = G::NGRP == 1 || grp == 1;
    // s = Z t on row r = m - 2 - LD (rel - 2 - 2 LD = r - j0)
    if (gb1 && (!CHK || (rel - 2 - 2 * LD >= 0 && rel - 2 - 2 * LD < nrows)) && col_ok) {
      constexpr int KR = K - 2 - LD;
      const T *tr = tt + pmod(KR, G::NTT) * G::WTC;
      T acc = tr[R];
#pragma unroll
      for (int s = 0; s < NZ; ++s) {
        // row r - dy(s) holds the column whose Z entry reaches (col, r)
        const int kz = KR - P::dy(s);
        const unsigned char *bz = gb[gback(K, 2 + LD + P::dy(s))];
        const T *trow = tt + pmod(kz, G::NTT) * G::WTC;
        acc = fma(fld(bz, G::OFF_Z + s * FBZ, pmod(kz, RB), G::WZ)[G::HZ - P::dx(s)], trow[R - P::dx(s)], acc);
      }
      const int r = mlo + rel - 2 - LD;
      if (edge) {
#pragma unroll
        for (int w = 0; w < (NW > 0 ? NW : 1); ++w) {
          const int target = P::wdx(w) - 1 - P::wcol(w);   // 0 or 1
          if (col == target) acc = fma(zwrap[(size_t)r * NW + w], tr[R - P::wdx(w)], acc);
        }
      }
      const T rv = rn[pmod(KR, G::NRN) * G::WRC + 2 * R];
      const size_t ro = (size_t)r * pitch;
      cs.put(s_out + ro, acc);
      if (kind != K2_APPLY) cs.put(rout + ro, rv);
      dot0.add(acc, rv);
      dot1.add(rv, rv);
    }
    // t on row mt = m - 1 (rel - 1 - LD = mt - j0)
    if (ga && (!CHK || (rel - 1 - LD >= 0 && rel - 1 <= nr1))) {
      const unsigned char *bz = gb[gback(K, 1)];
      const int mt = mlo + rel - 1;
      T *tm = tt + pmod(K - 1, G::NTT) * G::WTC;
      if (G::NCG <= G::WTC || lt < G::WTC) tm[0] = tcol<K - 1>(bz, 0, mt);
      if (lt < G::WTC - G::NCG) tm[G::NCG] = tcol<K - 1>(bz, G::NCG, mt);   // columns past the threads
    }
    bool got = true, waited = false;
    // r' on row m over [i0-2R, i0+TX+2R)
    if (ga && (!CHK || rel <= nr1)) {
      if constexpr (I == 0) {
        got = mbar_wait_or_abort(&full[fslot], fpar, timeout_ns, abort);
        waited = true;
        if (++fslot == (uint32_t)NSG) { fslot = 0; fpar ^= 1u; }
      }
      const T *Rr = fld(gb[0], G::OFF_R, I, G::WR), *Qr = fld(gb[0], G::OFF_Q, I, G::WR);
      T *rnm = rn + (K & (G::NRN - 1)) * G::WRC;
      constexpr int k0 = G::HR - 2 * R;
      if (G::NCG <= G::WRC || lt < G::WRC) {
        T v = Rr[k0];
        if (kind == K2_ITER) v = fma(-alpha, Qr[k0], v);
        rnm[0] = v;
      }
      if (lt < G::WRC - G::NCG) {
        T v2 = Rr[k0 + G::NCG];
        if (kind == K2_ITER) v2 = fma(-alpha, Qr[k0 + G::NCG], v2);
        rnm[G::NCG] = v2;
      }
    }
    if constexpr (I == 0) {
      if (!compute_sync_and<G::NC>(got)) return false;
    } else {
      compute_sync<G::NC>();
    }
    if (waited) ++nseen;
    // row m - 2 - LD is finished: at the last row of its group, release the group
    if constexpr (pmod(K - 1 - LD, RB) == 0) {
      if (!CHK || rel - 2 - LD >= 0) {
        mbar_arrive_if(&empty[eslot], tid == 0);
        if (++eslot == (uint32_t)NSG) eslot = 0;
        ++nrel;
      }
    }
    return true;
  }

  // All steps of the unit (rel = 0 .. nrows + 2 LD + 1); releases the unit's groups.
  // Blocks of 8 steps inside [2 + 2 LD, nr1] (all phases active) skip the checks.
  __device__ __forceinline__ bool run() {
    const int last = nrows + 2 * LD + 1;
    for (int b = 0; b <= last; b += 8) {
      if (b >= 2 + 2 * LD && b + 7 <= nr1) {
#define PCG_K2_STEADY(K) \
  if (!step<K, false>(b + K)) return false;
        PCG_K2_STEADY(0) PCG_K2_STEADY(1) PCG_K2_STEADY(2) PCG_K2_STEADY(3)
        PCG_K2_STEADY(4) PCG_K2_STEADY(5) PCG_K2_STEADY(6) PCG_K2_STEADY(7)
#undef PCG_K2_STEADY
        continue;
      }
#define PCG_K2_STEP(K) \
  if (b + K > last) break; \
  if (!step<K, true>(b + K)) return false;
      PCG_K2_STEP(0) PCG_K2_STEP(1) PCG_K2_STEP(2) PCG_K2_STEP(3)
      PCG_K2_STEP(4) PCG_K2_STEP(5) PCG_K2_STEP(6) PCG_K2_STEP(7)
#undef PCG_K2_STEP
    }
    for (; nrel < ng; ++nrel) {
      mbar_arrive_if(&empty[eslot], tid == 0);
      if (++eslot == (uint32_t)NSG) eslot = 0;
    }
    return true;
  }
};

template <typename T, int TX, class P, int KIND, bool DYN>
__global__ void __launch_bounds__(K2Geom<T, TX, P>::NT, K2Geom<T, TX, P>::MINB) k_precond(KParams p) {
  using G = K2Geom<T, TX, P>;
  constexpr int R = P::R, LD = P::LD, NZ = P::NZ, NW = P::NW;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = align128(smem_raw);
  const RingCtl<G::NSG> rc(base);
  T *rn = reinterpret_cast<T *>(rc.ring + (size_t)G::NSG * G::GROUP);
  T *tt = rn + (size_t)G::NRN * G::WRC;
  double *red = reinterpret_cast<double *>(tt + (size_t)G::NTT * G::WTC);
  constexpr int kind = KIND;
  const int tid = threadIdx.x;
  LaunchState *ls = p.ls;

  if (p.guard && blockIdx.x == 0 && tid == 0) loop_guard(ls, p);
  if (tid == 0) {
    for (int s = 0; s < G::NSG; ++s) { mbar_init(&rc.full[s], 1); mbar_init(&rc.empty[s], 1); }
    rc.ctl[CTL_ABORT] = 0; rc.ctl[CTL_ARMED] = 0; rc.ctl[CTL_SEEN] = 0; rc.ctl[CTL_FLAG] = 0;
    rc.ctl[CTL_PUB] = 0; rc.ctl[CTL_CONS] = 0;
    fence_mbar_init();
  }
  __syncthreads();

  auto skip_unit = [&](const SolveState *st) {
    return kind != K2_APPLY && *(const volatile int32_t *)&st->done != 0;
  };

  if (tid >= G::NC) {
    // ---- producer warp
    auto setup = [&](int ui, int f, FieldCopy &c, bool &has, int &mlo, int &ng, int &u_end) -> bool {
      const Unit un = p.units[ui];
      const GridDev<T> *gdp = reinterpret_cast<const GridDev<T> *>(p.grids) + un.g;
      u_end = gdp->u_off + gdp->n_units;
      if (skip_unit(gdp->st)) return false;
      const int i0 = un.sx * TX, j0 = gdp->own0 + un.sy * gdp->ty;
      const int rend = min(j0 + gdp->ty, gdp->own1);
      const int mhi = rend + LD - 1;
      mlo = j0 - LD;
      ng = (mhi - mlo + G::RB) / G::RB;
      const int rsel = (kind == K2_APPLY) ? 0 : gdp->st->rsel;
      const TensorMapBytes *tm = gdp->tm;
      auto mk = [&](const T *plane, int tmi, int col, int off, int w) {
        c.src = reinterpret_cast<const char *>(plane + i0 + col);
        c.tmap = tm ? (const void *)(tm + tmi) : nullptr;
        c.pitch_b = (int64_t)gdp->pitch * (int64_t)sizeof(T);
        c.x = 128 / (int)sizeof(T) + i0 + col;
        c.dst = (uint32_t)off;
        c.bytes = (uint32_t)(G::RB * w * (int)sizeof(T));
      };
      has = true;
      if (f == 0) mk(gdp->r[rsel], rsel ? TM_WR_R1 : TM_WR_R0, -G::HR, G::OFF_R, G::WR);
      else if (f == 1) { mk(gdp->q, TM_WR_Q, -G::HR, G::OFF_Q, G::WR); has = kind == K2_ITER; }
      else if (f - 2 < NZ) mk(gdp->z[f - 2], TM_WZ_Z0 + f - 2, -G::HZ, G::OFF_Z + (f - 2) * G::fb(G::WZ), G::WZ);
      else if (f - 2 == NZ) mk(gdp->dinv, TM_WZ_DI, -G::HZ, G::OFF_DI, G::WZ);
      else has = false;
      return true;
    };
    const uint32_t gq =
        produce_all<G::NSG, G::RB, DYN>(p, rc.ring, G::GROUP, rc.full, rc.empty, rc.ctl, setup);
    if (tid == G::NC) rc.ctl[CTL_ARMED] = (int)gq;
  } else {
    // ---- compute threads
    uint32_t gbase = 0, seen = 0;
    bool aborted = false;
    for (int k = 0, ui = compute_unit<DYN, G::NC>(p, rc.ctl, 0, 0); ui >= 0;
         ui = compute_unit<DYN, G::NC>(p, rc.ctl, ++k, ui)) {
      const Unit un = p.units[ui];
      const GridDev<T> *gdp = reinterpret_cast<const GridDev<T> *>(p.grids) + un.g;
      SolveState *st = gdp->st;
      if constexpr (!DYN) {                  // (claimed units of skipped grids are never queued)
        if (skip_unit(st)) {
          ui = skip_grid(ui, gdp->u_off + gdp->n_units) - (int)gridDim.x;
          continue;
        }
      }
      const int nx = gdp->nx, ny = gdp->ny;
      const int i0 = un.sx * TX, j0 = gdp->own0 + un.sy * gdp->ty;
      const int rend = min(j0 + gdp->ty, gdp->own1);
      const int mlo = j0 - LD, mhi = rend + LD - 1;
      const int ng = (mhi - mlo + G::RB) / G::RB;
      double acc0 = 0.0, acc1 = 0.0;
      const int rsel = (kind == K2_APPLY) ? 0 : st->rsel;
      if (!aborted) {
        K2Unit<T, TX, P, KIND> cx;
        cx.tid = tid; cx.grp = tid / G::NCG; cx.lt = tid - cx.grp * G::NCG;
        cx.rn = rn + cx.lt; cx.tt = tt + cx.lt; cx.full = rc.full; cx.empty = rc.empty;
        cx.abort = &rc.ctl[CTL_ABORT]; cx.timeout_ns = p.timeout_ns;
        cx.begin(rc.ring, gbase);
        cx.nx = nx; cx.ny = ny; cx.mlo = mlo; cx.j0 = j0; cx.i0 = i0; cx.nr1 = mhi - mlo;
        cx.nrows = rend - j0; cx.ng = ng; cx.pitch = gdp->pitch; cx.col = i0 + cx.lt;
        cx.col_ok = cx.lt < TX && cx.col < nx;
        cx.cs.init(cx.col, nx, cx.col_ok);
        cx.alpha = (kind == K2_ITER) ? (T)st->alpha : (T)0;
        cx.rout = gdp->r[rsel ^ 1]; cx.s_out = gdp->s; cx.zwrap = gdp->zwrap;
        // the strips holding the first or last columns apply the periodic side table
        // (a warp vote: the compiler then treats the flag as uniform across the warp)
        cx.edge = __any_sync(0xffffffffu, NW > 0 && (i0 < 2 * R + 2 || i0 + TX + 2 * R + 2 > nx));
        if (!cx.run()) aborted = true;
        seen = gbase + (uint32_t)cx.nseen;
        acc0 = cx.dot0.total();
        acc1 = cx.dot1.total();
      }
      gbase += ng;
      if (aborted && tid == 0) { rc.ctl[CTL_ABORT] = 1; flag_timeout(st); }
      if (kind == K2_APPLY) continue;
      if (unit_reduce2<G::NC>(acc0, acc1, gdp->partial, un.u, gdp->n_units, &st->cnt2, red, &rc.ctl[CTL_FLAG])) {
        if (tid == 0) {
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
    if (tid == 0) rc.ctl[CTL_SEEN] = (int)seen;
  }
  __syncthreads();
  drain_groups<G::NSG>(rc, p.timeout_ns);
  if constexpr (DYN) launch_exit(ls);
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
  const int j0 = gd.own0 + un.sy * gd.ty, rend = min(j0 + gd.ty, gd.own1);
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
  const int j0 = gd.own0 + un.sy * gd.ty, rend = min(j0 + gd.ty, gd.own1);
  if (col < gd.nx) {
    for (int r = j0; r < rend; ++r) {
      const size_t ro = (size_t)r * gd.pitch;
      const T v = gd.a[ro + col] > (T)0 ? (T)user[(size_t)(r + gd.row_off) * gd.nx + col] : (T)0;
      store_dup(dst + ro, col, gd.nx, v);
    }
  }
}

// Mixed precision, refinement step: the binary64 residual r (plane r[rsel] of
// the binary64 grid) scaled by a power of two becomes the binary32 right-hand
// side b of the inner solve, whose solution x and directions d start at zero
// (cleared here at the same points). scale 0: the scale the refinement step
// chose on the device (SolveState::scale of the binary64 grid).
// (one block of strip-width threads per unit of the binary64 planes)
static __global__ void k_residual_to_f32(const GridDev<double> *g64, const GridDev<float> *g32, const Unit *units,
                                  double scale) {
  const int TX = (int)blockDim.x;
  const Unit un = units[blockIdx.x];
  const GridDev<double> &a = g64[un.g];
  const GridDev<float> &f = g32[un.g];
  if (*(volatile int32_t *)&a.st->retired) return;
  const int col = un.sx * TX + threadIdx.x;
  const int j0 = a.own0 + un.sy * a.ty, rend = min(j0 + a.ty, a.own1);
  const double *r = a.r[a.st->rsel];
  const double sc = scale != 0.0 ? scale : a.st->scale;
  float *b = const_cast<float *>(f.b);
  if (col < a.nx)
    for (int j = j0; j < rend; ++j) {
      const size_t ro = (size_t)j * f.pitch;
      store_dup(b + ro, col, a.nx, (float)(r[(size_t)j * a.pitch + col] * sc));
      store_dup(f.x + ro, col, a.nx, 0.0f);
      store_dup(f.d[0] + ro, col, a.nx, 0.0f);
      store_dup(f.d[1] + ro, col, a.nx, 0.0f);
    }
}

// Mixed precision, refinement step: x += e / scale with e the binary32 inner
// solution (x plane of the binary32 grid); the update is done in binary64.
// inv_scale 0: 1 / SolveState::scale of the binary64 grid.
// (one block of strip-width threads per unit of the binary64 planes)
static __global__ void k_correct_f64(const GridDev<double> *g64, const GridDev<float> *g32, const Unit *units,
                              double inv_scale) {
  const int TX = (int)blockDim.x;
  const Unit un = units[blockIdx.x];
  const GridDev<double> &a = g64[un.g];
  const GridDev<float> &f = g32[un.g];
  if (*(volatile int32_t *)&a.st->retired || *(volatile int32_t *)&f.st->retired) return;
  const int col = un.sx * TX + threadIdx.x;
  const int j0 = a.own0 + un.sy * a.ty, rend = min(j0 + a.ty, a.own1);
  const double inv = inv_scale != 0.0 ? inv_scale : 1.0 / a.st->scale;
  if (col < a.nx)
    for (int j = j0; j < rend; ++j) {
      double *xr = a.x + (size_t)j * a.pitch;
      store_dup(xr, col, a.nx, fma(to_f64(f.x[(size_t)j * f.pitch + col]), inv, xr[col]));
    }
}

// padded plane -> user [ny][nx] (land = 0), over every cell
template <typename T, typename U>
__global__ void k_unpack(const GridDev<T> *gdp, U *user, int which) {
  const GridDev<T> &gd = *gdp;
  const T *srcp = which == 0 ? gd.x : which == 1 ? gd.s : which == 2 ? gd.q : gd.r[0];
  // the solution of b = 0 is x = 0 whatever the x plane holds
  const bool zero = which == 0 && gd.st->bzero != 0;
  // the own rows only (all rows of a whole grid)
  const size_t n = (size_t)gd.nx * (size_t)(gd.own1 - gd.own0);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int j = gd.own0 + (int)(e / gd.nx), i = (int)(e % gd.nx);
    const size_t o = (size_t)j * gd.pitch + i;
    user[(size_t)(j + gd.row_off) * gd.nx + i] = (gd.a[o] > (T)0 && !zero) ? (U)srcp[o] : (U)0;
  }
}

}  // namespace pcg
