// Host-side steps 1-2 of Sec. II.B: fill-reducing ordering and symbolic
// factorisation, producing the multifrontal layout the kernels run on.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace pexsi {

// One front per supernode K: its columns [first[K], first[K+1]) (s_K of them,
// new numbering) followed by its off-diagonal row structure C_K (r_K rows,
// ascending, all > the last column of K). The front is an m_K x m_K
// column-major block, m_K = s_K + r_K, local row index: 0..s_K-1 for the
// supernode's own columns, s_K + t for the t-th row of C_K.
struct Symbolic {
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> perm;    // perm[new] = old
  std::vector<int32_t> iperm;   // iperm[old] = new

  int32_t nsuper = 0;
  std::vector<int32_t> first;     // nsuper + 1
  std::vector<int64_t> rptr;      // nsuper + 1, offsets into rows / rel
  std::vector<int32_t> rows;      // C_K rows (new numbering)
  std::vector<int32_t> rel;       // position of each C_K row in the parent's front
  std::vector<int32_t> parent;    // supernodal elimination tree (Eq. parent), -1 = root
  std::vector<int32_t> height;    // 0 for leaves, 1 + max(children) otherwise
  std::vector<int64_t> front_off; // nsuper + 1, element offsets of the fronts in one pole's pool

  // Per CSC entry e: pool offset of its lower-triangle position (row >= col
  // in the new numbering) inside its front, and whether e is that lower copy.
  std::vector<int64_t> entry_pos;
  std::vector<uint8_t> entry_lower;
  // The mirror of entry_pos across the front's diagonal: the upper-triangle
  // position of the same pair of rows (LDU fronts store both triangles).
  std::vector<int64_t> entry_pos_up;

  int32_t nlevels = 0;
  std::vector<std::vector<int32_t>> level_fronts;  // fronts per height, big first

  // statistics (see pexsi_plan_stats)
  int64_t nnz_L = 0, front_elems = 0, max_front = 0, max_width = 0;
  int32_t s(int K) const { return first[K + 1] - first[K]; }
  int32_t r(int K) const { return int32_t(rptr[K + 1] - rptr[K]); }
  int32_t m(int K) const { return s(K) + r(K); }
};

struct FlopCounts {
  double factor_gemm = 0, selinv_gemm = 0, diag = 0, gather_bytes = 0;
};

// Validates the CSC pattern and runs the analysis. Returns 0 or a negative
// PEXSI_ERR_* code with a message in err.
int analyse(int64_t n, const int64_t* colptr, const int32_t* rowind, const int32_t* perm_or_null,
            int leaf_cols, bool amalgamate, Symbolic& out, std::string& err);

// Algorithmic flop counts of one pole for panel width b (complex arithmetic,
// 8 real flops per multiply-add).
FlopCounts count_flops(const Symbolic& sym, int b);

}  // namespace pexsi
