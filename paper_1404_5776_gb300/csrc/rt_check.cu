// Structural check of a block product's triple list (host code only).
//
// Every block-product kernel trusts its triple list: each output item owns
// one output block and is its only writer (so no two warps store to the same
// block, and the mirrored lower blocks of an upper-only product are never
// items), and each (a, b) pair indexes a stored block of A and of B inside
// the operand arrays.  This file states that contract as a check over host
// copies of the patterns and the list, for debugging and for tests: it is
// what a device-side bounds assert would test, done once per list instead of
// once per load.
#include <string>
#include <vector>

#include "rt_internal.cuh"

namespace rt {

namespace {

bool fail(std::string* why, const std::string& msg) {
  if (why) *why = msg;
  return false;
}

// rowptr from 0, non-decreasing; columns in range and strictly ascending in a
// row; symmetric ((i,j) present iff (j,i) present).  Fills the row of every block.
bool check_pattern(const char* name, int n, const int32_t* rp, const int32_t* col, std::vector<int32_t>& rowof,
                   std::string* why) {
  if (n < 0) return fail(why, "negative atom count");
  if (rp[0] != 0) return fail(why, std::string(name) + ": rowptr[0] != 0");
  for (int i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return fail(why, std::string(name) + ": rowptr decreases at row " + std::to_string(i));
  const int64_t nnzb = rp[n];
  rowof.assign((size_t)nnzb, 0);
  for (int i = 0; i < n; ++i)
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
      rowof[(size_t)q] = i;
      if (col[q] < 0 || col[q] >= n)
        return fail(why, std::string(name) + ": column out of range in row " + std::to_string(i));
      if (q > rp[i] && col[q] <= col[q - 1])
        return fail(why, std::string(name) + ": columns not strictly ascending in row " + std::to_string(i));
    }
  for (int i = 0; i < n; ++i)
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
      const int j = col[q];
      int32_t lo = rp[j], hi = rp[j + 1];
      while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (col[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= rp[j + 1] || col[lo] != i)
        return fail(why, std::string(name) + ": not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")");
    }
  return true;
}

// |row i of X ∩ row j of Y| (both ascending)
int64_t intersect(const int32_t* xrp, const int32_t* xcol, int i, const int32_t* yrp, const int32_t* ycol, int j) {
  int32_t p = xrp[i], pe = xrp[i + 1], q = yrp[j], qe = yrp[j + 1];
  int64_t n = 0;
  while (p < pe && q < qe) {
    if (xcol[p] < ycol[q]) ++p;
    else if (ycol[q] < xcol[p]) ++q;
    else {
      ++n;
      ++p;
      ++q;
    }
  }
  return n;
}

}  // namespace

bool check_triples_host(int n, const int32_t* a_rp, const int32_t* a_col, bool a_dag, const int32_t* b_rp,
                        const int32_t* b_col, bool b_dag, const int32_t* c_rp, const int32_t* c_col, bool upper_only,
                        int64_t n_items, const int32_t* item_blk, const int64_t* ptr, const int32_t* ab,
                        int64_t n_triples, int64_t* bad_item, std::string* why) {
  if (bad_item) *bad_item = -1;
  std::vector<int32_t> arow, brow, crow;
  if (!check_pattern("P_A", n, a_rp, a_col, arow, why) || !check_pattern("P_B", n, b_rp, b_col, brow, why) ||
      !check_pattern("P_C", n, c_rp, c_col, crow, why))
    return false;
  const int64_t nnzb_a = a_rp[n], nnzb_b = b_rp[n], nnzb_c = c_rp[n];
  // one item per output block (per block with col >= row for upper-only
  // products), in block order: every output block has exactly one writer
  int64_t expected = 0;
  for (int64_t q = 0; q < nnzb_c; ++q) {
    if (upper_only && c_col[q] < crow[(size_t)q]) continue;
    if (expected >= n_items || item_blk[expected] != q) {
      if (bad_item) *bad_item = expected < n_items ? expected : -1;
      return fail(why, "output block " + std::to_string(q) + " has no item (or items out of block order)");
    }
    ++expected;
  }
  if (expected != n_items) return fail(why, "more items than output blocks");
  if (n_items == 0) return n_triples == 0 ? true : fail(why, "triples without items");
  if (ptr[0] != 0) return fail(why, "ptr[0] != 0");
  if (ptr[n_items] != n_triples) return fail(why, "ptr[n_items] != n_triples");
  for (int64_t t = 0; t < n_items; ++t) {
    if (bad_item) *bad_item = t;
    if (ptr[t + 1] < ptr[t]) return fail(why, "ptr decreases");
    const int32_t qc = item_blk[t];
    const int i = crow[(size_t)qc], j = c_col[qc];
    int prev_k = -1;
    for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) {
      const int32_t a = ab[2 * e], b = ab[2 * e + 1];
      if (a < 0 || a >= nnzb_a) return fail(why, "A block index out of range");
      if (b < 0 || b >= nnzb_b) return fail(why, "B block index out of range");
      // op(A)_ik is the stored block (i,k), or (k,i) for A^dagger
      const int ra = arow[(size_t)a], ca = a_col[a];
      if ((a_dag ? ca : ra) != i) return fail(why, "A block is not in the output's row");
      const int k = a_dag ? ra : ca;
      // op(B)_kj is the stored block (k,j), or (j,k) for B^dagger
      const int rb = brow[(size_t)b], cb = b_col[b];
      if ((b_dag ? rb : cb) != j || (b_dag ? cb : rb) != k) return fail(why, "B block does not match (k, j)");
      if (k <= prev_k) return fail(why, "k not strictly ascending");
      prev_k = k;
    }
    // complete: one triple per k with (i,k) in P_A and (k,j) in P_B (symmetric patterns)
    if (ptr[t + 1] - ptr[t] != intersect(a_rp, a_col, i, b_rp, b_col, j)) return fail(why, "triples missing");
  }
  if (bad_item) *bad_item = -1;
  return true;
}

}  // namespace rt

rt_status rt_check_triples(int32_t n_atoms, const int32_t* a_rowptr, const int32_t* a_col, int32_t a_dag,
                           const int32_t* b_rowptr, const int32_t* b_col, int32_t b_dag, const int32_t* c_rowptr,
                           const int32_t* c_col, int32_t upper_only, int64_t n_items, const int32_t* item_blk,
                           const int64_t* ptr, const int32_t* ab, int64_t n_triples, int64_t* bad_item) {
  if (bad_item) *bad_item = -1;
  if (n_atoms < 0 || n_items < 0 || n_triples < 0 || !a_rowptr || !b_rowptr || !c_rowptr || !ptr) return RT_EINVAL;
  if ((a_rowptr[n_atoms] > 0 && !a_col) || (b_rowptr[n_atoms] > 0 && !b_col) || (c_rowptr[n_atoms] > 0 && !c_col) ||
      (n_items > 0 && !item_blk) || (n_triples > 0 && !ab))
    return RT_EINVAL;
  try {
    return rt::check_triples_host(n_atoms, a_rowptr, a_col, a_dag != 0, b_rowptr, b_col, b_dag != 0, c_rowptr, c_col,
                                  upper_only != 0, n_items, item_blk, ptr, ab, n_triples, bad_item, nullptr)
               ? RT_OK
               : RT_EINTERNAL;
  } catch (...) {
    return RT_EINTERNAL;
  }
}
