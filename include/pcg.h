/*
 * pcg.h -- C ABI of libpcg: AINV-preconditioned conjugate gradient for the
 * ocean free-surface elliptic system on one NVIDIA B300 (sm_103a).
 *
 * The method is that of Cuomo, De Michele, Farina and Chinnici, "A PCG
 * implementation of an elliptic kernel in an ocean global circulation model
 * based on GPU libraries" (2012):
 *   - the operator is the five-point system of Section 3, Eq. 9 on the
 *     natural ordering (west->east fastest, then south->north), in its SPD
 *     form, over wet points only, east-west periodic, north/south closed, plus
 *     the positive mass shift that the D^{n+1} term of Section 2, Eq. 2 adds
 *     to the diagonal;
 *   - the preconditioner is the factored approximate inverse of Section 3,
 *     M^-1 = Z D^-1 Z^T (Z unit upper triangular), built by conjugate
 *     orthogonalisation restricted to a sparsity pattern;
 *   - the solver is Algorithm 1 (FSAI-PCG), with the new direction
 *     d = s + beta d, stopping when ||r|| / ||b|| <= rtol.
 *
 * Conventions for every entry point:
 *   - Return value: a pcg_status (0 = PCG_OK). No C++ exception crosses this
 *     boundary. pcg_last_error_message() returns a thread-local description
 *     of the last failure in the calling thread.
 *   - Grid fields are row-major [ny][nx] (i = 0..nx-1 east-west, periodic;
 *     j = 0..ny-1 south-north). Vectors b and x use the same layout in
 *     binary64; entries on land are ignored on input and written as 0.
 *   - Vector pointers may be device pointers or host pointers (pageable or
 *     pinned); host buffers are copied through the handle's staging buffer on
 *     the given stream. The caller owns every buffer it passes.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Solves (pcg_solve, pcg_solve_batched) are enqueued on that
 *     stream and return at once; their x and statistics are valid after
 *     pcg_sync. The one-operand applies synchronise the stream before
 *     returning.
 *   - A handle owns all device memory it allocates; it is not thread-safe
 *     (one thread at a time). The solver server is thread-safe.
 */
#ifndef PCG_H
#define PCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PCG_OK = 0,
  PCG_EINVAL = 1,      /* invalid argument: sizes, null pointers, negative or non-finite coefficients */
  PCG_ENOMEM = 2,      /* device or host allocation failed */
  PCG_EBUDGET = 3,     /* solver server: admission refused by the HBM budget */
  PCG_ENOTCONV = 4,    /* max_iter reached: x holds the last iterate, stats are filled */
  PCG_EBREAKDOWN = 5,  /* non-positive pivot in the AINV build, (d, q) <= 0, or NaN/Inf in the iteration */
  PCG_ETIMEOUT = 6,    /* a bounded device wait or a server wait gave up */
  PCG_ECUDA = 7,       /* a CUDA runtime call failed */
  PCG_ECANCELLED = 8   /* solver server: the request was cancelled before it ran */
} pcg_status;

/* Problem definition (Section 3, Eq. 8-9; Section 2, Eq. 2).
 * c_e[j*nx+i]: coefficient of the face between (i,j) and ((i+1) mod nx, j).
 * c_n[j*nx+i]: coefficient of the face between (i,j) and (i,j+1); the last
 *              row's values are ignored.
 * A face touching a land cell carries no flux, whatever its value.
 * shift[j*nx+i]: diagonal mass term, > 0 on wet cells.
 * A_kk = shift_k + sum of the wet faces of k; A_km = -c_face.
 * All pointers are host pointers; the data is copied during ainv_setup. */
typedef struct {
  int32_t nx, ny;
  const uint8_t *wet;     /* [ny][nx], nonzero = ocean */
  const double *c_e;      /* [ny][nx], >= 0, finite */
  const double *c_n;      /* [ny][nx], >= 0, finite */
  const double *shift;    /* [ny][nx], > 0 and finite on wet cells */
} pcg_grid;

/* Sparsity pattern of Z (column k may hold rows m <= k of):
 *   PCG_PAT_TRIL_A  -- the lower part of the pattern of A (the k's west and
 *                      south neighbours, plus the periodic east neighbour of
 *                      the last column); Section 3's incomplete inverse
 *                      factorisation on a fixed pattern.
 *   PCG_PAT_TRIL_A2 -- the lower part of the pattern of A^2 (points within two
 *                      steps through wet cells).
 *   PCG_PAT_FULL    -- dense; reserved for the CPU oracle, rejected here.
 *   PCG_PAT_BAND_T  -- the paper's own choice (Section 3, pattern-selection
 *                      steps 1-6): Z from the east-west tridiagonal part T of
 *                      A, upper bandwidth band_q.
 *   PCG_PAT_DIAG    -- Z = I, D = diag(A): the diagonal (Jacobi) preconditioner
 *                      of Section 3, Eqs. 10-12. */
typedef enum {
  PCG_PAT_TRIL_A = 0,
  PCG_PAT_TRIL_A2 = 1,
  PCG_PAT_FULL = 2,
  PCG_PAT_BAND_T = 3,
  PCG_PAT_DIAG = 4
} pcg_pattern;

typedef struct {
  int32_t pattern;     /* pcg_pattern */
  double drop_tol;     /* drop |z_mk| sqrt(a_mm / a_kk) < drop_tol after every update; 0 = keep all */
  int32_t band_q;      /* PCG_PAT_BAND_T only: upper bandwidth q, 1..8 */
  int32_t tile_x;      /* device strip width in points: 64, 128, or a width whose preconditioner pass
                          fills whole warps (tril(A^2): 60 or 92 binary64 / 124 binary32; tril(A): 62 or
                          124 binary64 / 124 binary32), applied to the precisions that have it (the other
                          keeps its default); 0 = chosen per precision (binary64: 92 for tril(A^2) on grids
                          of 700 columns or more, 124 for tril(A) on grids of 2048 columns or more, else
                          60 / 62) */
  int32_t tile_y;      /* device strip height in rows, 4..256; 0 = chosen per precision at setup: the height
                          (4..128) minimising a model of the two loop launches' slowest CTA / SM over the
                          grid's wet strips and the resident CTAs (a shape tuned earlier wins) */
} ainv_opts;

typedef enum { PCG_FP64 = 0, PCG_MIXED = 1 } pcg_precision;

typedef struct {
  double rtol;         /* stop when ||r|| / ||b|| <= rtol (2-norm over wet points) */
  int32_t max_iter;    /* cap on inner iterations in total; <= 0 means the number of wet points */
  int32_t prec;        /* pcg_precision. PCG_MIXED: binary32 inner PCG inside a binary64
                          iterative-refinement loop (binary64 outer residual, x update and
                          inner dot-product accumulation) */
  double inner_rtol;   /* PCG_MIXED: relative tolerance of an inner solve (default 1e-5 if <= 0); once the
                          reduction still needed, rtol / relres, is >= inner_rtol / 10, the inner solve asks
                          for half of it instead (floor inner_rtol / 10) */
  int32_t max_outer;   /* PCG_MIXED: cap on refinement steps (default 30 if <= 0) */
  int32_t use_x0;      /* nonzero: x holds the initial guess on entry; zero: start from x = 0 */
  int32_t max_replace; /* FP64: restarts from the true residual when it fails rtol on exit (default 3 if < 0) */
} pcg_opts;

typedef struct {
  int32_t iters;        /* inner iterations (all refinement steps together) */
  int32_t outer_iters;  /* refinement steps (PCG_MIXED) or 1 + restarts (PCG_FP64) */
  int32_t status;       /* pcg_status of the solve */
  int32_t replacements; /* true-residual restarts taken */
  double relres;        /* recursive ||r|| / ||b|| at exit (binary64 outer residual in PCG_MIXED) */
  double true_relres;   /* ||b - A x|| / ||b|| computed on the device in binary64 at exit */
  double seconds;       /* wall time of the call */
} pcg_stats;

typedef struct pcg_handle pcg_handle;

/* Validate the grid, assemble A, build Z and D on the host by left-looking
 * conjugate orthogonalisation (Section 3; the paper builds its factor serially
 * on the CPU, Section 4), and upload A, Z, D^-1 to the device in the packed
 * strip layout. On success *out owns all device memory of this grid.
 * Errors: PCG_EINVAL (nx < 4, nx < 5 with PCG_PAT_TRIL_A2, ny < 1, null
 * pointers, negative or non-finite coefficients, shift <= 0 on a wet cell,
 * PCG_PAT_FULL, band_q out of range), PCG_EBREAKDOWN (non-positive pivot),
 * PCG_ENOMEM, PCG_ECUDA. */
int ainv_setup(const pcg_grid *grid, const ainv_opts *opts, void *cuda_stream, pcg_handle **out);

/* Solve A x = b (Algorithm 1 with its stopping rule): enqueue the whole solve
 * on cuda_stream and return without waiting for it. b: [ny][nx] binary64; x:
 * [ny][nx] binary64, read as the initial guess when opts->use_x0, written
 * with the solution (land = 0). opts may be NULL (rtol 1e-10, FP64).
 * The solve runs on the device from start to end: the PCG iterations, the
 * true-residual check at exit and the restarts from the true residual
 * (PCG_FP64), or the refinement steps (PCG_MIXED), are decided by device
 * kernels inside one CUDA graph launch, with no host round trip. x and *stats
 * (stats may be NULL; otherwise it must stay valid until then) are valid after
 * pcg_sync(h), which returns the solve's status: PCG_OK, PCG_ENOTCONV (x holds
 * the last iterate), PCG_EBREAKDOWN, PCG_ETIMEOUT. This call returns PCG_OK once
 * the solve is enqueued, or an error found before (PCG_EINVAL, PCG_ENOMEM,
 * PCG_ECUDA).
 * One solve may be in flight per handle: a call on a handle whose previous
 * solve has not been synchronised first waits for it (as pcg_sync does), and so
 * do the other entry points that use the handle. Host buffers go through the
 * handle's device staging buffer, copied on the handle's own copy stream and
 * ordered against cuda_stream by events, so that they overlap other work on
 * cuda_stream (another handle's solve; see pcg_clone). A device or pageable
 * host b may be reused as soon as the call returns (a pageable one is staged
 * at the call); a pinned host b must stay unchanged until pcg_sync(h). A
 * pageable host x makes the call wait for the solve (the copy into pageable
 * memory completes synchronously), a pinned one does not.
 * Without conditional CUDA graphs (or with PCG_LOOP_CHUNKED set) the solve is
 * done by a host-driven loop before the call returns; pcg_sync then only
 * reports it. */
int pcg_solve(pcg_handle *h, const double *b, double *x, const pcg_opts *opts, pcg_stats *stats,
              void *cuda_stream);

/* Solve nbatch independent systems, one per handle (each handle at most
 * once), advancing all of them in lock-step: every device launch covers the
 * work of all unconverged members, and converged members drop out. Each
 * member's result equals what pcg_solve gives for it alone (same kernels, same
 * per-grid reduction order). Enqueued like pcg_solve; stats ([nbatch], may be
 * NULL) and every x are valid after pcg_sync on any member, which returns
 * PCG_OK if every member converged, else the first failing member's status.
 * The plans and graph of a batch are kept for later calls on the same handles
 * (the four most recent batches). */
int pcg_solve_batched(pcg_handle *const *hs, int32_t nbatch, const double *const *b, double *const *x,
                      const pcg_opts *opts, pcg_stats *stats, void *cuda_stream);

/* Wait for the solve enqueued on h (pcg_solve or pcg_solve_batched): its work
 * on its stream, not what was queued there after it, and the copies of its
 * solutions into host buffers. Fill its statistics and return its status (see
 * pcg_solve_batched for a batch). With nothing in flight, returns the status of
 * h's last synchronised solve (PCG_OK if none). PCG_ECUDA if the device
 * reported an error. */
int pcg_sync(pcg_handle *h);

/* A second handle of the same grid and factor: a copy of src's host grid, Z
 * and D, and strips, with device planes, state and staging of its own (no
 * factorisation). Since one solve may be in flight per handle, two handles of
 * one grid let a caller keep two solves in flight, e.g. alternate right-hand
 * sides between them so that one solve's host copies overlap the other's
 * iterations. The paper has no counterpart. src is only read (it may have a
 * solve in flight). Errors: PCG_EINVAL (null pointers), PCG_ENOMEM, PCG_ECUDA.
 * Free the copy with pcg_free. */
int pcg_clone(const pcg_handle *src, void *cuda_stream, pcg_handle **out);

/* q = A v on the device kernels of the iteration (Section 3, Eq. 9).
 * Returns PCG_OK, PCG_EINVAL, PCG_ECUDA, or PCG_ETIMEOUT when a bounded device
 * wait gave up (q is then incomplete). */
int pcg_spmv(pcg_handle *h, const double *v, double *q, void *cuda_stream);

/* q = A v like pcg_spmv, but without allocating anything. The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate device memory where they call it -- an ocean model whose own memory
 * manager claims the whole device at start-up, or code that runs under a fixed
 * device-memory budget that a hidden cudaMalloc would break.
 * Its scratch (the packed v and q planes and the grid descriptor) lives in a
 * file-scope device array of 2^21 binary64 values per plane (about 32 MiB in
 * all), which every GPU that loads the library keeps until the process exits.
 * v and q must be device pointers ([ny][nx] binary64). Grids whose padded
 * plane ((ny + 4) rows times the strip-padded row pitch) exceeds 2^21 values are
 * rejected with PCG_EINVAL and a message giving the limit. The first call on a
 * device looks up the array's device address with that device current, so make
 * that first call before any stream capture. All calls share the one array and
 * each call overwrites it (clearing it first): calls that overlap on the GPU --
 * from different streams or threads -- race and must not be issued. The call
 * synchronises cuda_stream before returning. Errors: PCG_EINVAL, PCG_ECUDA,
 * PCG_ETIMEOUT (a bounded device wait gave up; q is incomplete). */
int pcg_spmv_noalloc(pcg_handle *h, const double *v, double *q, void *cuda_stream);

/* s = Z D^-1 Z^T r on the device kernels of the iteration (the preconditioning
 * step of Algorithm 1). Same errors as pcg_spmv. */
int pcg_precond_apply(pcg_handle *h, const double *r, double *s, void *cuda_stream);

/* Export the library's own factor for comparison: for each wet point k in
 * natural order, D[k] and the off-diagonal entries of column k of Z.
 * Entries are reported as (row index m, value) pairs; rows/vals hold room
 * for 8 entries per column ([n_wet][8], unused entries have row = -1).
 * n_wet_out receives the number of wet points. Any output may be NULL to
 * query n_wet only. */
int pcg_ainv_export(const pcg_handle *h, int32_t *n_wet_out, double *D, int32_t *rows, double *vals);

/* Build the library's factor on the host only (no device needed) and export
 * it as pcg_ainv_export does. n_wet_out receives the number of wet points;
 * D, rows, vals must hold nx*ny, 8*nx*ny and 8*nx*ny entries (an upper bound
 * of the wet count). Same errors as ainv_setup, without PCG_ECUDA. */
int ainv_factor_host(const pcg_grid *grid, const ainv_opts *opts, int32_t *n_wet_out, double *D, int32_t *rows,
                     double *vals);

/* Test hook for the bounded device waits: runs one preconditioner launch of
 * the grid in which the first row copy of work unit `unit` is deliberately
 * never issued, with every device wait limited to timeout_ms. The waiting CTA
 * gives up, records PCG_ETIMEOUT in the grid's device state and returns; the
 * call returns that recorded status (PCG_ETIMEOUT when the guard works). The
 * handle stays usable. No GPU fault is involved. */
int pcg_debug_wait_timeout(pcg_handle *h, int32_t unit, double timeout_ms, void *cuda_stream);

/* The binary32 kernels of the mixed-precision mode (the inner iterations of
 * the refinement loop) on one operand, for checking them alone:
 *   op 0: out = A v (Section 3, Eq. 9 in SPD form), the stencil kernel;
 *   op 1: out = Z D^-1 Z^T v (the preconditioning step of Algorithm 1), the
 *         preconditioner kernel.
 * v and out are [ny][nx] binary64 (host or device); v is rounded to binary32
 * on the way in, the binary32 result widened on the way out; land entries of
 * out are 0. Builds the handle's binary32 planes on first use. Returns PCG_OK,
 * PCG_EINVAL (NULL argument or op not 0/1), PCG_ENOMEM or PCG_ECUDA. */
int pcg_apply_f32(pcg_handle *h, int32_t op, const double *v, double *out, void *cuda_stream);

/* Strip-shape autotuner (batching, tile shapes chosen by measurement): for
 * precision prec (PCG_FP64: the binary64 planes; PCG_MIXED: the binary32
 * planes of the inner iterations) times the two loop kernels of h on strips
 * of 64, 128 or the whole-warp widths (tile_x) columns by 8, 16, 32 or 64 rows (ten iterations each, on a
 * right-hand side of ones), rebuilds h's planes with the best shape and
 * returns it in tile_x, tile_y (either may be NULL). objective 0: the
 * shortest kernel time of the grid alone (a single solve); objective 1: the
 * smallest share of the GPU, kernel time x min(units, resident CTAs) /
 * resident CTAs (the grid as one member of a batch or of a server's mix).
 * The result is kept for the process, keyed by (nx, ny, pattern, band_q,
 * prec, objective): a later call for the same key applies it without timing,
 * and ainv_setup without explicit tiles uses the objective-0 shapes.
 * Overwrites the handle's last solution. Not thread-safe for h.
 * Returns PCG_OK, PCG_EINVAL, PCG_ENOMEM or PCG_ECUDA. */
int pcg_autotune(pcg_handle *h, int32_t prec, int32_t objective, int32_t *tile_x, int32_t *tile_y,
                 void *cuda_stream);

/* The strip shape (columns, rows) of h's planes of precision prec. */
int pcg_tiles(pcg_handle *h, int32_t prec, int32_t *tile_x, int32_t *tile_y);

/* Measurement entry point: loads b, runs the init kernels, then `iters` PCG
 * iterations as individual launches of the stencil kernel and of the
 * preconditioner kernel, each bracketed by CUDA events on cuda_stream.
 * Writes the mean duration of one launch of each (milliseconds). prec =
 * PCG_FP64 times the binary64 kernels; PCG_MIXED times the binary32 kernels of
 * the inner solves (on b rounded to binary32). The iterations are real (the
 * state advances as in a solve); x is not returned. Errors: PCG_EINVAL,
 * PCG_ECUDA. */
int pcg_profile_kernels(pcg_handle *h, const double *b, int32_t iters, int32_t prec, double *ms_stencil,
                        double *ms_precond, void *cuda_stream);

/* Measurement entry point (no counterpart in the paper): the binary64
 * fused multiply-add rate of the current GPU, the unit that bounds the binary64
 * iteration on this part. Runs one warm-up and then `launches` launches of a
 * kernel in which every thread of one full wave of resident blocks advances 8
 * independent FMA chains, times them with CUDA events on cuda_stream and
 * writes the rate in TFLOP/s (2 flops per FMA) to *tflops and the mean launch
 * time to *ms_per_launch (may be NULL). Allocates and frees a small device
 * buffer. Errors: PCG_EINVAL (tflops NULL or launches <= 0), PCG_ECUDA. */
int pcg_fp64_fma_rate(int32_t launches, double *tflops, double *ms_per_launch, void *cuda_stream);

/* Number of kernel launches this library has issued since it was loaded,
 * counting every kernel run inside a loop graph. */
uint64_t pcg_kernel_launches(void);

/* Device bytes held by this handle (A, Z, D^-1, work vectors, scratch). */
size_t pcg_resident_bytes(const pcg_handle *h);

/* Number of wet unknowns of this handle's grid. */
int32_t pcg_n_wet(const pcg_handle *h);

/* Release the handle and its device memory. NULL is accepted. */
void pcg_free(pcg_handle *h);

const char *pcg_status_string(int status);
const char *pcg_last_error_message(void);

/* --------------------------------------------------- row-band sharding */

/* The layout in which one large grid is split over several GPUs: contiguous
 * bands of rows of about equal wet count. The paper has no counterpart (it runs
 * one GPU); the iteration is Algorithm 1 unchanged, whose two reductions per
 * iteration become the only global steps besides the exchange of band-edge
 * rows. pcg_band_plan computes the bands of a mask on the host: row0[b] ..
 * row0[b + 1] - 1 are band b's rows (row0 has nbands + 1 entries, row0[0] = 0,
 * row0[nbands] = ny), each band at least *halo rows tall; *halo is the number of
 * a neighbour's rows a band reads: max(1, LD) with LD = 2 for
 * PCG_PAT_TRIL_A2, 1 for PCG_PAT_TRIL_A, 0 otherwise. Errors: PCG_EINVAL (NULL
 * argument, nbands < 1, or fewer than nbands * halo rows). */
int pcg_band_plan(int32_t nx, int32_t ny, const uint8_t *wet, int32_t pattern, int32_t nbands, int32_t *row0,
                  int32_t *halo);

typedef struct pcg_shard pcg_shard;

/* Split the grid of h (binary64 planes) into nbands >= 2 bands on the current
 * GPU: each band gets planes for its rows and *halo rows of each neighbour,
 * with A, Z and D^-1 taken from h's factor (built once for the whole grid),
 * and every kernel of the solve runs over all bands' own rows in one launch,
 * sharing one reduction state (on several GPUs these would be per-rank
 * partial sums and two allreduces per iteration). The rows a band reads from
 * a neighbour are refreshed by an exchange kernel after the kernel that wrote
 * them (on several GPUs: sends and receives of the same row blocks). h must
 * outlive the shard and not be retiled while it exists. Errors: PCG_EINVAL,
 * PCG_ENOMEM, PCG_ECUDA. */
int pcg_shard_create(pcg_handle *h, int32_t nbands, void *cuda_stream, pcg_shard **out);

/* The bands of a shard: *nbands, row0[nbands + 1] and *halo (any may be NULL). */
int pcg_shard_bands(const pcg_shard *sh, int32_t *nbands, int32_t *row0, int32_t *halo);

/* Solve A x = b over the bands (binary64, Algorithm 1 with the true-residual
 * check and restarts decided on the device, as pcg_solve). b and x are device
 * pointers, [ny][nx] binary64 (x read as x0 when opts->use_x0). Synchronises
 * cuda_stream; returns the solve status and fills stats (may be NULL). */
int pcg_shard_solve(pcg_shard *sh, const double *b, double *x, const pcg_opts *opts, pcg_stats *stats,
                    void *cuda_stream);

void pcg_shard_free(pcg_shard *sh);

/* ---------------------------------------------------------------- serving */

typedef struct {
  size_t hbm_budget_bytes;   /* admission limit on the device bytes of registered grids + right-hand-side buffers */
  int32_t max_slots;         /* requests that may be on the device at once (1..256) */
  int32_t chunk_iters;       /* iterations run between admission/retirement points */
  pcg_opts solve;            /* options applied to every request */
} pcg_server_opts;

typedef struct {
  uint64_t submitted, completed, failed, rejected;
  double p50_latency_ms, p99_latency_ms, mean_latency_ms;  /* submission -> completion */
  double solves_per_s;       /* completed / (last completion - first submission) */
  int32_t in_flight, queued;
  size_t hbm_used_bytes;
} pcg_server_stats;

typedef struct pcg_server pcg_server;

/* Continuous-batching solver server. A scheduler thread keeps up to max_slots
 * requests on the device, advancing all of them together in chunks of
 * chunk_iters iterations; between chunks it retires converged requests and
 * admits queued ones, so requests that arrive while others run join the next
 * chunk. Each grid's requests run in submission order (a timestep depends on
 * the previous solution); with warm starts, each request starts from the last
 * solution of its grid. */
int solver_server_create(const pcg_server_opts *opts, pcg_server **out);

/* Register a grid; the handle stays owned by the caller, must outlive the
 * server, and must not be used outside it while the server runs. In a mixed
 * precision server the grid's binary32 planes are built here and counted.
 * Fails with PCG_EBUDGET if the grid's resident bytes do not fit. */
int solver_server_register(pcg_server *s, pcg_handle *h, int32_t *grid_id);

/* Queue a solve of grid grid_id with right-hand side b ([ny][nx], host or
 * device; copied into a device buffer of the grid's pool before this call
 * returns) writing the solution to x_out ([ny][nx], host or device, written
 * when the request completes). If warm_start is nonzero the solve starts from
 * the grid's last solution: an ocean model solves the free-surface system once
 * per time step, and the previous step's surface is the natural initial guess
 * (the paper's x0 of Algorithm 1 is a previous state too), which is why this
 * argument, absent from a plain queue interface, is part of the call. done (may be NULL) is called from the scheduler
 * thread on completion. A new pool buffer counts against the HBM budget;
 * PCG_EBUDGET if it does not fit (the request is not queued). */
int solver_server_submit(pcg_server *s, int32_t grid_id, const double *b, double *x_out, int32_t warm_start,
                         void (*done)(void *user, const pcg_stats *stats), void *user, uint64_t *req_id);

/* Wait for one request; fills stats (may be NULL) and returns its status,
 * or PCG_ETIMEOUT if timeout_ms (< 0 = forever) expires first. The statistics
 * (iterations, residuals, latency from submission) are returned here because a
 * request's caller, not the server, decides what to do with a solve that did
 * not converge. */
int solver_server_wait(pcg_server *s, uint64_t req_id, int32_t timeout_ms, pcg_stats *stats);

/* Cancel a request that has not yet been admitted to the device. */
int solver_server_cancel(pcg_server *s, uint64_t req_id);

int solver_server_stats(pcg_server *s, pcg_server_stats *out);

/* Stop the scheduler (pending requests complete with PCG_ECANCELLED) and free the server. */
void solver_server_destroy(pcg_server *s);

#ifdef __cplusplus
}
#endif

#endif /* PCG_H */
