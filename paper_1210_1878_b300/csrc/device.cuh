// Device kernels of libpcg (sm_103a).
//
// Data layout. Every field of a grid lives in a padded row-major plane:
// element (i, j) is at base[j * pitch + i] for j in [-GY, ny + GY) and i in
// [-GX, pitch - GX). Rows j < 0 and j >= ny are zero. Columns -GHOST..-1 and
// nx..nx+GHOST-1 hold periodic copies of columns nx-GHOST..nx-1 and 0..GHOST-1
// (every writer of a column near the edge also writes its copies), so a halo
// read across the periodic face is a plain read. Land cells hold zeros in every
// field (A's coefficients and diagonal, Z, D^-1 and all vectors), so land never
// needs a mask: it stays zero through every operation.
//
// Work units. A grid is cut into strips TX columns wide and TY rows tall; only
// strips holding a wet cell become units. A persistent CTA of TX compute
// threads (plus a producer warp) handles a unit at a time, thread t owning
// column i0 + t. It marches north one row at a time while the producer warp
// streams the input fields, several rows per copy, into a ring of
// shared-memory slots (tensor or bulk asynchronous copies, completion counted
// on an mbarrier per slot), running on into the CTA's next unit. Values needed from
// neighbouring rows (the stencil's north/south points, the rows Z^T pulls from
// and the rows Z pushes to) are computed once per row into small shared rings,
// so every point's floating-point work is done once; only the few halo columns
// at a strip's sides are recomputed.
//
// Reductions. Each unit writes its partial sums to its own slot; the last CTA
// of a grid (arrival counter) adds the partials in unit order, so the result
// does not depend on scheduling or on what else shares the launch. That CTA
// also advances the grid's scalar recurrence (alpha, beta, rho, the stopping
// test) in the grid's device-resident state.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pcg {

constexpr int GY = 2;          // zero rows below and above
constexpr int GHOST = 4;       // periodic copies kept on each side

// kinds of launch of the stencil kernel
enum { K1_ITER = 0, K1_RESID_INIT = 1, K1_RESID_CHECK = 2, K1_SPMV = 3 };
// kinds of launch of the preconditioner kernel
enum { K2_ITER = 0, K2_INIT = 1, K2_APPLY = 2 };

struct SolveState {
  double rho, alpha, pending, beta;   // recurrence scalars; pending = alpha not yet applied to x
  double rr, bb, dq, rr_true;         // last reductions
  double rtol;
  int32_t iter, max_iter, status, done;
  int32_t dsel, rsel, bzero, retired;   // retired: set once the result is final
  uint32_t cnt1, cnt2, pad2, pad3;    // arrival counters of the two kernels
  // Control of a whole solve, decided on the device between passes (the
  // true-residual restarts of a binary64 solve; the refinement steps of a
  // mixed-precision solve, kept in the binary64 state).
  int32_t final_status;               // pcg_status once the result is final, else -1
  int32_t pad4;
  int32_t replacements, max_replace;  // restarts taken / allowed
  double scale;                       // mixed: power of two scaling the residual into binary32
  double relres64;                    // mixed: binary64 ||b - A x|| / ||b|| of the last refinement step
  double inner_rtol;                  // mixed: tolerance of an inner solve far from the finish
  int32_t inner_iters, inner_solves;  // mixed: inner iterations and inner solves so far
  int32_t budget, max_outer;          // mixed: cap on inner iterations in total, on refinement steps
};

struct LaunchState {
  int32_t active;          // grids of the launch not yet done
  int32_t launches;        // loop-body executions so far
  int32_t max_launches;    // hard cap on body executions (a runaway guard)
  int32_t stop;            // set when the loop must end
  cudaGraphConditionalHandle cond;
  uint64_t t0_ns;          // device time of the first loop body (0 until then)
  uint64_t budget_ns;      // wall-clock cap on the loop (a runaway guard)
  int32_t timed_out;
  int32_t cond_cleared;    // the loop condition has been cleared in this launch
  int32_t bodies_total;    // loop-body executions over every pass of a solve (launch count)
  int32_t passes;          // outer passes of a solve (restarts / refinement steps + 1)
  uint32_t claim_next;     // next unit of a running claiming launch (0 between launches)
  uint32_t claim_exit;     // CTAs of the running claiming launch that have finished (0 between launches)
};

// A CUtensorMap as the kernels see it: 128 opaque bytes, 64-byte aligned.
struct alignas(64) TensorMapBytes {
  unsigned long long w[16];
};

// Tensor maps of a grid (RB > 1 streaming), one per plane and box width:
// WS = TX + 2H, WT = TX, WE = TX + H of the stencil kernel; WR, WZ of the
// preconditioner kernel.
enum {
  TM_WS_S = 0, TM_WS_D0, TM_WS_D1, TM_WS_X,
  TM_WT_CN, TM_WT_A, TM_WT_X, TM_WT_B,
  TM_WE_CE,
  TM_WR_R0, TM_WR_R1, TM_WR_Q,
  TM_WZ_DI, TM_WZ_Z0,
  TM_COUNT = TM_WZ_Z0 + 8
};

template <typename T>
struct GridDev {
  int32_t nx, ny, pitch, ty;
  int32_t n_units, n_wrap;
  int32_t u_off;           // index of this grid's first unit in the launch's unit list
  int32_t pad1;
  const T *ce, *cn, *a, *dinv;
  const T *z[8];
  const T *zwrap;          // [ny][n_wrap]
  T *x, *s, *q;
  T *r[2], *d[2];
  const T *b;
  double *partial;         // [n_units][2]
  SolveState *st;
  const TensorMapBytes *tm;   // [TM_COUNT] or null (one row per copy)
  // A row band of a larger grid (sharded solve): local row j is row j + row_off
  // of the caller's [ny][nx] vectors, and rows [own0, own1) are the band's own
  // (the others are halo rows filled by the exchange). A whole grid: 0, 0, ny.
  int32_t row_off, own0, own1, pad2;
};

struct Unit {              // one strip of one grid
  int16_t g, sx;
  int16_t sy, pad;
  int32_t u;               // index of the unit within its grid
};

struct KParams {
  const void *grids;       // GridDev<T>[]
  const Unit *units;
  LaunchState *ls;
  int32_t kind;
  int32_t use_cond;        // 1 when launched inside the conditional loop graph
  int32_t guard;           // 1 for the first stencil launch of the loop body
  int32_t dbg_skip_unit;   // test hook: unit whose first row copy is never issued (-1: none)
  uint64_t timeout_ns;     // bound on every mbarrier wait
  int32_t n_units;         // units in the list; CTAs stride over them (persistent)
  int32_t pad;
};

}  // namespace pcg
