// Internal declarations shared by the host and device translation units of libpcg.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcg.h"

namespace pcg {

// ---------------------------------------------------------------- slots of Z
// Column k of Z is stored as a fixed set of "slots": slot o holds the entry
// Z[m, k] for the point m = k + offset(o) (periodic in i). Offsets that only
// occur through the periodic face (the last columns' east neighbours, which
// precede them in the natural ordering) are kept in a small per-row side table
// instead of full slot planes.
struct SlotSet {
  int n = 0;                 // number of slot planes
  int dx[16], dy[16];        // offset of each plane
  int n_wrap = 0;            // side-table entries per row
  // side-table entry w: column (nx - 1 - wcol[w]) holds row (wdx[w] - 1 - wcol[w]) mod nx, same j
  int wcol[4], wdx[4];
  int lower_rows = 0;        // max -dy over planes (rows below needed by Z^T)
  int reach = 0;             // max |dx| over planes and side-table offsets
};

SlotSet slot_set(int pattern, int band_q);

// Host result of the AINV build, wet-compressed (natural order).
struct HostFactor {
  int32_t n = 0;
  SlotSet slots;
  std::vector<double> d;          // [n]
  std::vector<double> z;          // [slots.n][n]
  std::vector<double> zwrap;      // [ny][slots.n_wrap]
};

struct HostGrid {
  int32_t nx = 0, ny = 0, n = 0;
  std::vector<int32_t> idx;       // [ny*nx] wet index or -1
  std::vector<int32_t> pi, pj;    // [n]
  std::vector<double> ce, cn;     // [ny*nx] face coefficients, 0 on faces touching land
  std::vector<double> diag;       // [n]
};

// Validate and assemble; returns a pcg_status and sets the error message.
int host_grid_build(const pcg_grid *g, int pattern, HostGrid &out, std::string &err);
// Left-looking AINV over the slot layout; returns a pcg_status.
int host_ainv(const HostGrid &G, int pattern, double tau, int band_q, HostFactor &F, std::string &err);

void set_error(const std::string &msg);

}  // namespace pcg
