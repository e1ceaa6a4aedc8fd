// Internal declarations of the GB300 density-matrix RT-TDDFT library.
//
// Data layout (device):
//   * one system = n_atoms atoms, every atom padded to the system's block size
//     B (1, 4 or 13); padded functions are decoupled (S = 1, H = D = K = 0 there),
//     so every product is exact on the unpadded part;
//   * a pattern = block-CSR over atoms (rowptr, col ascending, rowidx per block,
//     tmap = index of the transposed block, diag = index of (i,i));
//   * a matrix = values of its pattern's blocks, B*B row-major per block, as
//     double (real), double2 (complex FP64), float or float2 (FP32 mode);
//   * a product C = op(A) op(B) cut to P_C is described by a triple list:
//     items (output blocks) with ranges of (a_block, b_block) pairs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/rt.h"

namespace rt {

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
struct Error {
  rt_status code;
  std::string msg;
};

#define RT_CUDA_CHECK(expr)                                                          \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      throw ::rt::Error{RT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e) + \
                                      " at " + __FILE__ + ":" + std::to_string(__LINE__)}; \
    }                                                                                \
  } while (0)

#define RT_REQUIRE(cond, code, text)                        \
  do {                                                      \
    if (!(cond)) throw ::rt::Error{(code), std::string(text)}; \
  } while (0)

// ----------------------------------------------------------------------------
// device memory (allocator hook from the C ABI)
// ----------------------------------------------------------------------------
struct Allocator {
  rt_alloc_fn alloc = nullptr;
  rt_free_fn free = nullptr;
  void* user = nullptr;
  void* get(size_t bytes, cudaStream_t stream);
  void put(void* p, cudaStream_t stream);
};

// A device buffer owned by the context (freed in bulk at destroy).
struct Arena {
  Allocator* alloc = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<void*> blocks;
  size_t total = 0;
  void* get(size_t bytes);
  template <typename T>
  T* get_n(size_t n) {
    return static_cast<T*>(get(n * sizeof(T) + 16));
  }
  void release_all();
};

// ----------------------------------------------------------------------------
// patterns and triple lists
// ----------------------------------------------------------------------------
struct Pattern {
  double radius = 0.0;
  int n_atoms = 0;
  int64_t nnzb = 0;
  int32_t* rowptr = nullptr;  // [n_atoms+1]
  int32_t* col = nullptr;     // [nnzb]
  int32_t* rowidx = nullptr;  // [nnzb]
  int32_t* tmap = nullptr;    // [nnzb] index of (j,i)
  int32_t* diag = nullptr;    // [n_atoms] index of (i,i)
  std::vector<int32_t> h_rowptr, h_col;  // host copies (tests, maps)
};

struct Triples {
  int64_t n_items = 0;
  int64_t n_triples = 0;
  int32_t* item_blk = nullptr;  // [n_items] output block index in P_C
  int64_t* ptr = nullptr;       // [n_items+1]
  int2* ab = nullptr;           // [n_triples] (a block, b block)
};

// Row tiles of a triple list for the tensor-core products: up to TC_TILE
// consecutive items of one output block row; per tile the merged, ascending
// list of the A blocks its items use (one "entry" per distinct A block, i.e.
// per k of the row), with the B block each item multiplies it by (-1: the
// item has no triple with that k).
constexpr int TC_TILE = 8;
struct TileList {
  bool built = false;
  int64_t n_tiles = 0;
  int64_t n_entries = 0;
  int32_t* item0 = nullptr;  // [n_tiles] first item of the tile
  int32_t* nitem = nullptr;  // [n_tiles] items in the tile (1..TC_TILE)
  int64_t* uptr = nullptr;   // [n_tiles+1] entry range
  int32_t* ua = nullptr;     // [n_entries] A block of the entry
  int32_t* ub = nullptr;     // [n_entries][TC_TILE] B block per item slot, -1 = none
};

// Build P_r on the device (cell lists, minimum image, FP64 without contraction).
void build_pattern(Pattern& P, int n_atoms, const double* d_pos, const double* cell, double r,
                   Arena& arena, cudaStream_t st);
// Pattern from host block-CSR arrays (given S / H patterns).
void upload_pattern(Pattern& P, int n_atoms, const int32_t* rowptr, const int32_t* col, double r,
                    Arena& arena, cudaStream_t st);
// Triple list for C = op(A) op(B) cut to P_C (optionally only blocks with j >= i).
void build_triples(Triples& T, const Pattern& A, bool a_dag, const Pattern& B, bool b_dag,
                   const Pattern& C, bool upper_only, Arena& arena, cudaStream_t st);
// map[q] = index in `dst` of block q of `src` (or -1).
void build_block_map(int32_t* map, const Pattern& src, const Pattern& dst, cudaStream_t st);
// map[q] = index in `dst` of the transpose (j,i) of block q=(i,j) of `src` (or -1).
void build_transpose_map(int32_t* map, const Pattern& src, const Pattern& dst, cudaStream_t st);

// Row tiles of a triple list whose items are the blocks of P_C (or its upper
// blocks) in increasing order, each item's triples in increasing A block.
void build_tiles(TileList& tl, const Triples& T, const Pattern& C, Arena& arena, cudaStream_t st);

// exclusive scan of int64 counts (n+1 outputs, out[n] = total); returns total
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& arena, cudaStream_t st);

// Structural check of a triple list against its patterns (host arrays; the
// conditions of rt_check_triples).  False with the reason in *why on failure.
bool check_triples_host(int n, const int32_t* a_rp, const int32_t* a_col, bool a_dag, const int32_t* b_rp,
                        const int32_t* b_col, bool b_dag, const int32_t* c_rp, const int32_t* c_col, bool upper_only,
                        int64_t n_items, const int32_t* item_blk, const int64_t* ptr, const int32_t* ab,
                        int64_t n_triples, int64_t* bad_item, std::string* why);

// ----------------------------------------------------------------------------
// block products
// ----------------------------------------------------------------------------
enum Epilogue : int {
  EPI_STORE = 0,      // C = acc
  EPI_STORE_ACC = 1,  // C = acc; U[re or im] += coef * acc       (Taylor powers)
  EPI_TWO_I = 2,      // C = 2I - acc; resid += |I - acc|^2         (Hotelling)
  EPI_SANDWICH = 3,   // C upper = acc, mirror lower, hermitian diagonal (K' = M U^dagger)
  EPI_ADD = 4,        // C += acc                                     (delta form)
  EPI_DELTA_SANDWICH = 5,  // C = base + add + acc, mirrored (delta form, mixed precision)
};

struct GemmArgs {
  const Triples* tri;       // host view (counts)
  const int32_t* item_blk;
  const int64_t* ptr;
  const int2* ab;
  int64_t n_items;
  const void* A;
  const void* B;
  void* C;
  // EPI_STORE_ACC
  void* U;                  // complex accumulator (double2 / float2)
  const int32_t* umap;      // output block -> U block (nullptr = same index)
  double coef;
  int coef_imag;            // 0: add to real part, 1: to imaginary part
  // EPI_TWO_I / reductions
  double* red;              // per-item partial sums
  const int32_t* rowidx;    // P_C row index per block
  const int32_t* colidx;    // P_C col per block
  const int32_t* tmap;      // P_C transpose map
  const int32_t* bsize;     // true functions per atom (residual mask)
  // delta-sandwich extras (FP64 K base and M addend on P_K)
  const void* base;
  const void* addend;
  const int32_t* add_map;   // P_K block -> addend block
  unsigned long long* herm_max;  // max |K_ii - K_ii^dagger| bits
  const void* base2;        // reference split: FP64 R = U K_ref U^dagger - K_ref at the output block, or null
  const void* zero;         // a zero block (FP32 kernels stage it for missing triples)
  int* err;                 // device error word: the largest code of a bounded wait that gave up
                            // (1: wait expired, copies drained; 2: the drain expired too)
  long long wait_ns;        // budget of one bounded wait (FP32 kernels), nanoseconds
  // delta sandwich of the reference split with the field polynomial: R(E) =
  // sum_p E^p B_p evaluated per element (Horner, FP64) in place of base2
  const double2* const* rpoly;  // device table of B_0..B_rdeg (dense blocks on P_K), or null
  int rdeg;
  const double* poly_E;     // device address of the field value E
  void* kf32;               // delta sandwich: also write K' rounded to FP32 (the FP32 block layout;
                            // the B operand of the next step's first product), or null
  // launch shape of the FP32 complex products (the tuner's choices)
  int stages;               // 13-function kernel: stages per warp (0 = default 2, or 3)
  int persistent;           // 1: at most one resident wave of CTAs, each walking items with a grid stride
  const GemmArgs* grp;      // grouped launch: device array of per-product arguments, or null
  const int2* gitems;       // grouped launch: (product, item within it) of every item
  int a_planar;             // complex 13-function FP32: A (and the W written by the delta
                            // form) column-planar, the packed-FMA kernel
  // row tiles (tensor-core products)
  int64_t tl_n;
  const int32_t* tl_item0;
  const int32_t* tl_nitem;
  const int64_t* tl_uptr;
  const int32_t* tl_ua;
  const int32_t* tl_ub;
};

// Row stride of an FP32 block: 13-function blocks are padded to 13 x 16
// (16-byte aligned rows, the shared-memory layout of the FP32 kernels).
inline int rs32(int B) { return B == 13 ? 16 : B; }
inline int sb32(int B) { return B * rs32(B); }

// Complex 13-function FP32 products on the tensor cores (tcgen05, 3xTF32 split,
// FP32 accumulation of per-k partial sums) over row tiles (g.tl_*), with the
// epilogues EPI_STORE (and W = K + M) and EPI_DELTA_SANDWICH; false if `epi`
// is not one of them.
bool launch_gemm13_tc(Epilogue epi, const GemmArgs& g, cudaStream_t st);

// Launches; `cplx` selects complex values, `b_dag` conj-transposes B's blocks,
// `a_dag` A's blocks.  Element type by precision: FP64 double/double2, FP32 float/float2.
void launch_gemm(int B, bool fp32, bool cplx, bool a_dag, bool b_dag, Epilogue epi,
                 const GemmArgs& g, cudaStream_t st);

// ----------------------------------------------------------------------------
// elementwise / reductions
// ----------------------------------------------------------------------------
void launch_fill_zero(void* p, size_t bytes, cudaStream_t st);

}  // namespace rt
