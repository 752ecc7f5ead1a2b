// Allocation-free variant of the operator apply q = A v (pcg_spmv_noalloc).
//
// pcg_spmv packs v into one of the handle's padded work planes and writes q
// into another. This variant does the same with scratch that lives in a
// file-scope device array instead: the packed input plane, the packed output
// plane and the grid descriptor the kernels read. It calls no cudaMalloc,
// cudaFree or other allocating routine, so it can be used by callers that own
// all device memory themselves (an ocean model whose memory manager claims the
// whole device at start-up) or that run under a fixed device-memory budget
// where a hidden allocation at the point of the call would break it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "handle.cuh"

using namespace pcg;

namespace {

// Largest padded plane (elements) the static scratch can hold: 2^21 binary64
// values, i.e. grids with (ny + 4) * pitch <= 2,097,152 (for example up to
// 1442 x 1021 with 128-wide strips).
constexpr size_t kMaxPlaneElems = size_t(1) << 21;
constexpr size_t kHeaderBytes = 256;   // holds one GridDev<double>
static_assert(sizeof(GridDev<double>) <= kHeaderBytes, "grid descriptor does not fit the scratch header");

// Every GPU that loads the library keeps this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes + 2 * kMaxPlaneElems * sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. The first call
// on a device resolves it (cudaGetSymbolAddress) with that device current.
int scratch_address(void **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal out of range"); return PCG_EINVAL; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e));
      return PCG_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PCG_OK;
}

}  // namespace

extern "C" int pcg_spmv_noalloc(pcg_handle *h, const double *v, double *q, void *cuda_stream) {
  if (!h || !v || !q) { set_error("NULL argument"); return PCG_EINVAL; }
  if (!is_device_ptr(v) || !is_device_ptr(q)) { set_error("v and q must be device pointers"); return PCG_EINVAL; }
  handle_finish_pending(h);   // one piece of work in flight per handle
  const DevPlanes<double> &P = h->p64;
  if (P.plane_elems > kMaxPlaneElems) {
    set_error("grid too large for the allocation-free scratch: padded plane of " + std::to_string(P.plane_elems) +
              " values, limit " + std::to_string(kMaxPlaneElems));
    return PCG_EINVAL;
  }
  void *base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char *b8 = static_cast<unsigned char *>(base);
  double *plane_v = reinterpret_cast<double *>(b8 + kHeaderBytes);
  double *plane_q = plane_v + kMaxPlaneElems;
  const size_t origin = (size_t)GY * P.pitch + P.gx;   // element (0, 0) inside a plane

  // descriptor: the handle's coefficient planes, the scratch planes for v and q
  GridDev<double> gd = P.gd;
  // binary64 kernel 1 streams one row per copy straight from the plane
  // pointers below; tensor maps would name the handle's own planes
  if (P.ks.rb1 != 1) { set_error("allocation-free operator apply needs one-row streaming"); return PCG_EINVAL; }
  gd.tm = nullptr;
  gd.d[0] = plane_v + origin;
  gd.d[1] = plane_v + origin;
  gd.q = plane_q + origin;
  // the kernels record a bounded wait that gave up in the handle's state
  int rc_st = apply_status_clear(P.st, s);
  if (rc_st) return rc_st;
  CK(cudaMemcpyAsync(b8, &gd, sizeof(gd), cudaMemcpyHostToDevice, s));
  // the scratch keeps the previous call's contents: land strips, ghost rows and
  // columns must read zero
  CK(cudaMemsetAsync(plane_v, 0, P.plane_elems * sizeof(double), s));
  CK(cudaMemsetAsync(plane_q, 0, P.plane_elems * sizeof(double), s));
  if (P.n_units > 0) {
    KParams p{};
    p.grids = b8;
    p.units = P.units_dev;
    p.ls = h->ls;
    p.kind = K1_SPMV;
    p.dbg_skip_unit = -1;
    p.timeout_ns = default_timeout_ns();
    const double *vin = v;
    int which = 3;
    void *pack_args[] = {&p, (void *)&vin, &which};
    CK(cudaLaunchKernel(P.ks.pack, dim3(P.n_units), dim3(P.tx), pack_args, 0, s));
    note_launches(1);
    void *k_args[] = {&p};
    p.n_units = P.n_units;
    CK(cudaLaunchKernel(P.ks.k1[K1_SPMV], dim3(persistent_grid(P.ks, 1, P.n_units)), dim3(P.ks.tb), k_args, P.ks.smem1, s));
    note_launches(1);
  }
  const GridDev<double> *gdp = reinterpret_cast<const GridDev<double> *>(b8);
  double *qout = q;
  int which_out = 2;
  void *un_args[] = {(void *)&gdp, (void *)&qout, &which_out};
  const size_t n = (size_t)P.nx * P.ny;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
  CK(cudaLaunchKernel(P.ks.unpack, dim3(blocks > 0 ? blocks : 1), dim3(256), un_args, 0, s));
  note_launches(1);
  // synchronises s; PCG_ETIMEOUT if a wait of the stencil launch gave up
  return apply_status_read(P.st, s);
}
