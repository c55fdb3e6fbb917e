// Internal declarations shared by the host setup (C++) and the CUDA sources of libr3mg.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/r3mg.h"

namespace r3mg {

constexpr int kPad = 4;          // row entries padded to a multiple of 4 (16-byte vector loads)
constexpr int kMaxWindow = 65535;  // window indices are uint16

struct Error {
  r3mg_status status;
  std::string msg;
};

// Point- or cell-based agglomeration by R-tree bisection (Section 3; Section 4).
struct HostPartition {
  int64_t n = 0;
  int dim = 0, depth = 0, levels = 0;
  std::vector<int64_t> perm;                  // perm[k] = caller index of tree position k
  std::vector<int64_t> iperm;                 // iperm[caller index] = tree position
  std::vector<int64_t> leaf_off;              // 2^D + 1
  std::vector<std::vector<int64_t>> box_off;  // [l], l >= 1: nbox_l + 1 offsets in tree order
  std::vector<std::vector<double>> lo, hi;    // [l], l >= 1: nbox_l * dim MBR bounds
  int64_t nbox(int l) const { return (int64_t)box_off[l].size() - 1; }
};

// Block adjacency of a level (rows: boxes of that level).
struct HostPattern {
  std::vector<int64_t> ptr;  // nbox + 1
  std::vector<int64_t> nbr;  // sorted neighbour boxes
};

// Fine-level (level 0) windowed layout: rows in tree order, entries sorted by window index.
struct HostFineLayout {
  std::vector<int64_t> row_ptr;   // n + 1, padded to kPad
  std::vector<uint16_t> idx;      // window index of every stored entry (0 for padding)
  std::vector<int64_t> src;       // CSR position of every stored entry, -1 for padding
  std::vector<int64_t> diag_src;  // CSR position of the diagonal of each tree row
  std::vector<int32_t> win_off;   // per (box, slot): start of that neighbour's points in the window
  std::vector<int64_t> win_src;   // per (box, slot): first tree row of the neighbour's staged run
  std::vector<int32_t> win_size;  // per box: window length
  int32_t win_max = 0;
  int64_t nnz = 0;                // stored entries without padding
};

// Host-side steps (host_setup.cpp).
bool partition_points(int64_t n, int dim, const double* coords, int leaf, int levels, HostPartition& P, Error& err);
bool partition_cells(int64_t n, int dim, const double* coords, int64_t ncells, const int64_t* cell_ptr,
                     const int64_t* cell_pts, int leaf, int levels, HostPartition& P, Error& err);
void fine_pattern(const HostPartition& P, const int64_t* rowptr, const int32_t* colidx, HostPattern& pat);
void coarse_pattern(const HostPattern& fine, int fan, int64_t nbox_coarse, HostPattern& out);
bool fine_layout(const HostPartition& P, const HostPattern& pat, const int64_t* rowptr, const int32_t* colidx,
                 HostFineLayout& lay, Error& err);
bool validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx, Error& err);
void gll_nodes01(int p, double* z);
double tridiag_max_eig(const std::vector<double>& diag, const std::vector<double>& off);
double tridiag_kth_eig(const std::vector<double>& diag, const std::vector<double>& off, int j);
double max_coupled_distance(int64_t n, int dim, const double* coords, const int64_t* rowptr, const int32_t* colidx);

}  // namespace r3mg
