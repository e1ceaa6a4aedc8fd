// Neighbour lists, truncated output patterns and triple lists (set-up).
//
// Paper Sec. II.A: matrix elements between atoms beyond the cut-off radius are
// zero, so every matrix lives on a pattern P_r = {(i,j) : |R_i - R_j| < r}, and
// every product C = A B is evaluated only on its output pattern.  Atoms are
// stationary (Sec. V.A), so the patterns and the list of contributing block
// triples (i,k,j) of each product are built once here.
#include <algorithm>
#include <cmath>

#include "rt_internal.cuh"

namespace rt {

// ----------------------------------------------------------------------------
// memory
// ----------------------------------------------------------------------------
void* Allocator::get(size_t bytes, cudaStream_t stream) {
  void* p = nullptr;
  if (alloc) {
    p = alloc(bytes, (void*)stream, user);
    RT_REQUIRE(p != nullptr, RT_ENOMEM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{RT_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + ") failed: " + cudaGetErrorString(e)};
    }
  }
  return p;
}

void Allocator::put(void* p, cudaStream_t stream) {
  if (!p) return;
  if (free) free(p, (void*)stream, user);
  else cudaFree(p);
}

void* Arena::get(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* p = alloc->get(bytes, stream);
  blocks.push_back(p);
  total += bytes;
  return p;
}

void Arena::release_all() {
  for (void* p : blocks) alloc->put(p, stream);
  blocks.clear();
  total = 0;
}

// ----------------------------------------------------------------------------
// exclusive scan (int64), three-phase with recursion on block sums
// ----------------------------------------------------------------------------
static constexpr int SCAN_T = 512;

__global__ void k_scan_block(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                             int64_t* __restrict__ bsum, int64_t n) {
  __shared__ int64_t s[SCAN_T];
  int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
  int64_t v = (i < n) ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_T; off <<= 1) {
    int64_t t = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = s[SCAN_T - 1];
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ boff, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_set_total(int64_t* out, int64_t n, const int64_t* last_in) {
  // out[n] = out[n-1] + in[n-1]
  out[n] = (n > 0) ? out[n - 1] + last_in[0] : 0;
}

static void scan_rec(const int64_t* in, int64_t* out, int64_t n, Arena& arena, cudaStream_t st) {
  if (n <= 0) return;
  int64_t nb = (n + SCAN_T - 1) / SCAN_T;
  int64_t* bsum = arena.get_n<int64_t>(nb + 1);
  k_scan_block<<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, bsum, n);
  RT_CUDA_CHECK(cudaGetLastError());
  if (nb > 1) {
    int64_t* boff = arena.get_n<int64_t>(nb + 1);
    scan_rec(bsum, boff, nb, arena, st);
    k_scan_add<<<(unsigned)nb, SCAN_T, 0, st>>>(out, boff, n);
    RT_CUDA_CHECK(cudaGetLastError());
  }
}

int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& arena, cudaStream_t st) {
  // scratch from a private arena so repeated set-up scans do not accumulate
  Arena tmp;
  tmp.alloc = arena.alloc;
  tmp.stream = st;
  int64_t total = 0;
  try {
    scan_rec(in, out, n, tmp, st);
    if (n > 0) {
      k_set_total<<<1, 1, 0, st>>>(out, n, in + (n - 1));
    } else {
      RT_CUDA_CHECK(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    }
    RT_CUDA_CHECK(cudaGetLastError());
    RT_CUDA_CHECK(cudaMemcpyAsync(&total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RT_CUDA_CHECK(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    tmp.release_all();
    throw;
  }
  tmp.release_all();
  return total;
}

// ----------------------------------------------------------------------------
// neighbour lists
// ----------------------------------------------------------------------------
struct CellGrid {
  int nc[3];
  double lo[3];
  double w[3];
  int periodic;
  double L[3];
};

// Minimum-image squared distance; every operation rounded separately (no FMA).
__device__ __forceinline__ double d2_min_image(const double* __restrict__ pos, int i, int j,
                                               const CellGrid& g) {
  double d2 = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double dx = __dsub_rn(pos[3 * j + d], pos[3 * i + d]);
    if (g.periodic) {
      double n = rint(__ddiv_rn(dx, g.L[d]));
      dx = __dsub_rn(dx, __dmul_rn(g.L[d], n));
    }
    double t = __dmul_rn(dx, dx);
    d2 = (d == 0) ? t : __dadd_rn(d2, t);
  }
  return d2;
}

__device__ __forceinline__ int cell_coord(double x, double lo, double w, int nc) {
  int c = (int)floor((x - lo) / w);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_of(const double* __restrict__ pos, int n, CellGrid g, int32_t* __restrict__ cell,
                          int32_t* __restrict__ count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c0 = cell_coord(pos[3 * i + 0], g.lo[0], g.w[0], g.nc[0]);
  int c1 = cell_coord(pos[3 * i + 1], g.lo[1], g.w[1], g.nc[1]);
  int c2 = cell_coord(pos[3 * i + 2], g.lo[2], g.w[2], g.nc[2]);
  int c = (c0 * g.nc[1] + c1) * g.nc[2] + c2;
  cell[i] = c;
  atomicAdd(&count[c], 1);
}

__global__ void k_i32_to_i64(const int32_t* __restrict__ a, int64_t* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

__global__ void k_scatter_cells(int n, const int32_t* __restrict__ cell, const int64_t* __restrict__ start,
                                int32_t* __restrict__ cursor, int32_t* __restrict__ atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell[i];
  int p = atomicAdd(&cursor[c], 1);
  atoms[start[c] + p] = i;
}

// Visits every distinct neighbour cell of atom i's cell once (all cells along
// a dimension with fewer than 3 cells) and every atom j with d2 < r2.
template <bool FILL>
__global__ void k_neighbours(const double* __restrict__ pos, int n, CellGrid g, double r2,
                             const int32_t* __restrict__ cell, const int64_t* __restrict__ start,
                             const int32_t* __restrict__ atoms, int64_t* __restrict__ count,
                             const int32_t* __restrict__ rowptr, int32_t* __restrict__ col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell[i];
  int cc[3] = {c / (g.nc[1] * g.nc[2]), (c / g.nc[2]) % g.nc[1], c % g.nc[2]};
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    if (g.nc[d] < 3) {
      lo[d] = 0;
      hi[d] = g.nc[d] - 1;
    } else {
      lo[d] = cc[d] - 1;
      hi[d] = cc[d] + 1;
    }
  }
  int64_t k = 0;
  int32_t base = FILL ? rowptr[i] : 0;
  for (int x = lo[0]; x <= hi[0]; ++x) {
    int xx = x;
    if (xx < 0 || xx >= g.nc[0]) {
      if (!g.periodic) continue;
      xx = (xx + g.nc[0]) % g.nc[0];
    }
    for (int y = lo[1]; y <= hi[1]; ++y) {
      int yy = y;
      if (yy < 0 || yy >= g.nc[1]) {
        if (!g.periodic) continue;
        yy = (yy + g.nc[1]) % g.nc[1];
      }
      for (int z = lo[2]; z <= hi[2]; ++z) {
        int zz = z;
        if (zz < 0 || zz >= g.nc[2]) {
          if (!g.periodic) continue;
          zz = (zz + g.nc[2]) % g.nc[2];
        }
        int cn = (xx * g.nc[1] + yy) * g.nc[2] + zz;
        for (int64_t p = start[cn]; p < start[cn + 1]; ++p) {
          int j = atoms[p];
          if (d2_min_image(pos, i, j, g) < r2) {
            if (FILL) col[base + k] = j;
            ++k;
          }
        }
      }
    }
  }
  if (!FILL) count[i] = k;
}

// Sort each row's columns ascending: rank of each entry = number of smaller
// entries (entries of a row are distinct).  One block per row.
__global__ void k_sort_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ in,
                            int32_t* __restrict__ out) {
  extern __shared__ int32_t srow[];
  int i = blockIdx.x;
  int b = rowptr[i], e = rowptr[i + 1];
  int len = e - b;
  const int cap = 8192;
  bool use_smem = len <= cap;
  if (use_smem)
    for (int t = threadIdx.x; t < len; t += blockDim.x) srow[t] = in[b + t];
  __syncthreads();
  const int32_t* src = use_smem ? srow : in + b;
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    int v = src[t];
    int rank = 0;
    for (int u = 0; u < len; ++u) rank += (src[u] < v);
    out[b + rank] = v;
  }
}

__global__ void k_rowidx(const int32_t* __restrict__ rowptr, int n, int32_t* __restrict__ rowidx) {
  int i = blockIdx.x;
  if (i >= n) return;
  for (int q = rowptr[i] + threadIdx.x; q < rowptr[i + 1]; q += blockDim.x) rowidx[q] = i;
}

__device__ __forceinline__ int32_t find_in_row(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                               int i, int j) {
  int lo = rowptr[i], hi = rowptr[i + 1];
  while (lo < hi) {
    int mid = lo + ((hi - lo) >> 1);
    if (col[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  return (lo < rowptr[i + 1] && col[lo] == j) ? lo : -1;
}

__global__ void k_tmap_diag(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ rowidx, int64_t nnzb, int32_t* __restrict__ tmap,
                            int32_t* __restrict__ diag) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  int i = rowidx[q], j = col[q];
  tmap[q] = find_in_row(rowptr, col, j, i);
  if (i == j) diag[i] = (int32_t)q;
}

static void finish_pattern(Pattern& P, Arena& arena, cudaStream_t st) {
  int n = P.n_atoms;
  P.rowidx = arena.get_n<int32_t>(P.nnzb);
  P.tmap = arena.get_n<int32_t>(P.nnzb);
  P.diag = arena.get_n<int32_t>(n);
  RT_CUDA_CHECK(cudaMemsetAsync(P.diag, 0xff, sizeof(int32_t) * n, st));
  if (n > 0) k_rowidx<<<n, 128, 0, st>>>(P.rowptr, n, P.rowidx);
  if (P.nnzb > 0)
    k_tmap_diag<<<(unsigned)((P.nnzb + 255) / 256), 256, 0, st>>>(P.rowptr, P.col, P.rowidx, P.nnzb, P.tmap,
                                                                  P.diag);
  RT_CUDA_CHECK(cudaGetLastError());
  P.h_rowptr.resize(n + 1);
  P.h_col.resize(P.nnzb);
  RT_CUDA_CHECK(cudaMemcpyAsync(P.h_rowptr.data(), P.rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, st));
  if (P.nnzb)
    RT_CUDA_CHECK(cudaMemcpyAsync(P.h_col.data(), P.col, sizeof(int32_t) * P.nnzb, cudaMemcpyDeviceToHost, st));
  // every row must hold its diagonal block and the pattern must be symmetric
  std::vector<int32_t> h_tmap(P.nnzb), h_diag(n);
  if (P.nnzb)
    RT_CUDA_CHECK(cudaMemcpyAsync(h_tmap.data(), P.tmap, sizeof(int32_t) * P.nnzb, cudaMemcpyDeviceToHost, st));
  RT_CUDA_CHECK(cudaMemcpyAsync(h_diag.data(), P.diag, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  RT_CUDA_CHECK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) RT_REQUIRE(h_diag[i] >= 0, RT_EINVAL, "pattern lacks diagonal block of atom " + std::to_string(i));
  for (int64_t q = 0; q < P.nnzb; ++q) RT_REQUIRE(h_tmap[q] >= 0, RT_EINVAL, "pattern is not symmetric");
}

void build_pattern(Pattern& P, int n, const double* d_pos, const double* cell, double r, Arena& arena,
                   cudaStream_t st) {
  RT_REQUIRE(r > 0.0, RT_EINVAL, "radius must be positive");
  P.radius = r;
  P.n_atoms = n;
  CellGrid g;
  g.periodic = cell != nullptr;
  // host bounding box for open systems
  std::vector<double> hpos(3 * (size_t)n);
  RT_CUDA_CHECK(cudaMemcpyAsync(hpos.data(), d_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  RT_CUDA_CHECK(cudaStreamSynchronize(st));
  for (int d = 0; d < 3; ++d) {
    double lo = 0.0, span;
    if (g.periodic) {
      span = cell[d];
      g.L[d] = cell[d];
    } else {
      lo = hpos.empty() ? 0.0 : hpos[d];
      double hi = lo;
      for (int i = 0; i < n; ++i) {
        lo = std::min(lo, hpos[3 * i + d]);
        hi = std::max(hi, hpos[3 * i + d]);
      }
      span = (hi - lo) + 1e-9;
      g.L[d] = 0.0;
    }
    int nc = (int)std::floor(span / r);
    nc = std::max(1, std::min(nc, 1024));
    g.nc[d] = nc;
    g.lo[d] = lo;
    g.w[d] = span / nc;
  }
  int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  Arena tmp;
  tmp.alloc = arena.alloc;
  tmp.stream = st;
  try {
    int32_t* cellof = tmp.get_n<int32_t>(n);
    int32_t* ccount = tmp.get_n<int32_t>(ncell);
    int64_t* ccount64 = tmp.get_n<int64_t>(ncell);
    int64_t* cstart = tmp.get_n<int64_t>(ncell + 1);
    int32_t* cursor = tmp.get_n<int32_t>(ncell);
    int32_t* atoms = tmp.get_n<int32_t>(n);
    RT_CUDA_CHECK(cudaMemsetAsync(ccount, 0, sizeof(int32_t) * ncell, st));
    RT_CUDA_CHECK(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * ncell, st));
    int tb = 128;
    if (n > 0) k_cell_of<<<(n + tb - 1) / tb, tb, 0, st>>>(d_pos, n, g, cellof, ccount);
    k_i32_to_i64<<<(ncell + 255) / 256, 256, 0, st>>>(ccount, ccount64, ncell);
    RT_CUDA_CHECK(cudaGetLastError());
    exclusive_scan_i64(ccount64, cstart, ncell, tmp, st);
    if (n > 0) k_scatter_cells<<<(n + tb - 1) / tb, tb, 0, st>>>(n, cellof, cstart, cursor, atoms);
    double r2 = r * r;
    int64_t* rcount = tmp.get_n<int64_t>(n);
    int64_t* rstart = tmp.get_n<int64_t>(n + 1);
    if (n > 0)
      k_neighbours<false><<<(n + tb - 1) / tb, tb, 0, st>>>(d_pos, n, g, r2, cellof, cstart, atoms, rcount,
                                                            nullptr, nullptr);
    RT_CUDA_CHECK(cudaGetLastError());
    int64_t nnzb = exclusive_scan_i64(rcount, rstart, n, tmp, st);
    RT_REQUIRE(nnzb < (int64_t)INT32_MAX, RT_EINVAL, "pattern too large for 32-bit block indices");
    P.nnzb = nnzb;
    P.rowptr = arena.get_n<int32_t>(n + 1);
    // int64 -> int32 rowptr
    std::vector<int64_t> h64(n + 1);
    RT_CUDA_CHECK(cudaMemcpyAsync(h64.data(), rstart, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    RT_CUDA_CHECK(cudaStreamSynchronize(st));
    std::vector<int32_t> h32(n + 1);
    int maxlen = 0;
    for (int i = 0; i <= n; ++i) h32[i] = (int32_t)h64[i];
    for (int i = 0; i < n; ++i) maxlen = std::max(maxlen, h32[i + 1] - h32[i]);
    RT_CUDA_CHECK(cudaMemcpyAsync(P.rowptr, h32.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
    int32_t* unsorted = tmp.get_n<int32_t>(nnzb);
    P.col = arena.get_n<int32_t>(nnzb);
    if (n > 0)
      k_neighbours<true><<<(n + tb - 1) / tb, tb, 0, st>>>(d_pos, n, g, r2, cellof, cstart, atoms, nullptr,
                                                           P.rowptr, unsorted);
    RT_CUDA_CHECK(cudaGetLastError());
    size_t smem = (size_t)std::min(maxlen, 8192) * sizeof(int32_t);
    if (n > 0) k_sort_rows<<<n, 128, smem, st>>>(P.rowptr, unsorted, P.col);
    RT_CUDA_CHECK(cudaGetLastError());
    RT_CUDA_CHECK(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    tmp.release_all();
    throw;
  }
  tmp.release_all();
  finish_pattern(P, arena, st);
}

void upload_pattern(Pattern& P, int n, const int32_t* rowptr, const int32_t* col, double r, Arena& arena,
                    cudaStream_t st) {
  P.radius = r;
  P.n_atoms = n;
  RT_REQUIRE(rowptr[0] == 0, RT_EINVAL, "rowptr[0] must be 0");
  for (int i = 0; i < n; ++i) {
    RT_REQUIRE(rowptr[i + 1] >= rowptr[i], RT_EINVAL, "rowptr not monotone");
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      RT_REQUIRE(col[q] >= 0 && col[q] < n, RT_EINVAL, "column index out of range");
      if (q > rowptr[i]) RT_REQUIRE(col[q] > col[q - 1], RT_EINVAL, "columns not strictly ascending");
    }
  }
  P.nnzb = rowptr[n];
  P.rowptr = arena.get_n<int32_t>(n + 1);
  P.col = arena.get_n<int32_t>(P.nnzb);
  RT_CUDA_CHECK(cudaMemcpyAsync(P.rowptr, rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
  if (P.nnzb) RT_CUDA_CHECK(cudaMemcpyAsync(P.col, col, sizeof(int32_t) * P.nnzb, cudaMemcpyHostToDevice, st));
  finish_pattern(P, arena, st);
}

// ----------------------------------------------------------------------------
// block maps
// ----------------------------------------------------------------------------
__global__ void k_block_map(const int32_t* __restrict__ s_rowidx, const int32_t* __restrict__ s_col, int64_t nnzb,
                            const int32_t* __restrict__ d_rowptr, const int32_t* __restrict__ d_col, int transpose,
                            int32_t* __restrict__ map) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  int i = s_rowidx[q], j = s_col[q];
  map[q] = transpose ? find_in_row(d_rowptr, d_col, j, i) : find_in_row(d_rowptr, d_col, i, j);
}

void build_block_map(int32_t* map, const Pattern& src, const Pattern& dst, cudaStream_t st) {
  if (src.nnzb == 0) return;
  k_block_map<<<(unsigned)((src.nnzb + 255) / 256), 256, 0, st>>>(src.rowidx, src.col, src.nnzb, dst.rowptr,
                                                                   dst.col, 0, map);
  RT_CUDA_CHECK(cudaGetLastError());
}

void build_transpose_map(int32_t* map, const Pattern& src, const Pattern& dst, cudaStream_t st) {
  if (src.nnzb == 0) return;
  k_block_map<<<(unsigned)((src.nnzb + 255) / 256), 256, 0, st>>>(src.rowidx, src.col, src.nnzb, dst.rowptr,
                                                                   dst.col, 1, map);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ----------------------------------------------------------------------------
// triple lists
// ----------------------------------------------------------------------------
__global__ void k_item_flags(const int32_t* __restrict__ rowidx, const int32_t* __restrict__ col, int64_t nnzb,
                             int upper_only, int64_t* __restrict__ flag) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  flag[q] = (!upper_only || col[q] >= rowidx[q]) ? 1 : 0;
}

__global__ void k_item_compact(const int64_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t nnzb,
                               int32_t* __restrict__ item_blk) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  if (flag[q]) item_blk[pos[q]] = (int32_t)q;
}

// For output block (i,j): k runs over row i of P_A merged with row j of P_B
// (patterns are symmetric, so row j of P_B lists the k with (k,j) in P_B).
template <bool FILL>
__global__ void k_triples(const int32_t* __restrict__ item_blk, int64_t n_items,
                          const int32_t* __restrict__ c_rowidx, const int32_t* __restrict__ c_col,
                          const int32_t* __restrict__ a_rowptr, const int32_t* __restrict__ a_col,
                          const int32_t* __restrict__ a_tmap, int a_dag,
                          const int32_t* __restrict__ b_rowptr, const int32_t* __restrict__ b_col,
                          const int32_t* __restrict__ b_tmap, int b_dag,
                          int64_t* __restrict__ count, const int64_t* __restrict__ ptr, int2* __restrict__ ab) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  int q = item_blk[it];
  int i = c_rowidx[q], j = c_col[q];
  int pa = a_rowptr[i], ea = a_rowptr[i + 1];
  int pb = b_rowptr[j], eb = b_rowptr[j + 1];
  int64_t n = 0;
  int64_t base = FILL ? ptr[it] : 0;
  while (pa < ea && pb < eb) {
    int ka = a_col[pa], kb = b_col[pb];
    if (ka < kb) {
      ++pa;
    } else if (kb < ka) {
      ++pb;
    } else {
      if (FILL) {
        int a_blk = a_dag ? a_tmap[pa] : pa;  // op(A)_ik: A_ik, or (A_ki)^dagger
        int b_blk = b_dag ? pb : b_tmap[pb];  // op(B)_kj: B_kj, or (B_jk)^dagger
        ab[base + n] = make_int2(a_blk, b_blk);
      }
      ++n;
      ++pa;
      ++pb;
    }
  }
  if (!FILL) count[it] = n;
}

void build_triples(Triples& T, const Pattern& A, bool a_dag, const Pattern& B, bool b_dag, const Pattern& C,
                   bool upper_only, Arena& arena, cudaStream_t st) {
  Arena tmp;
  tmp.alloc = arena.alloc;
  tmp.stream = st;
  try {
    int64_t nnzb = C.nnzb;
    int64_t* flag = tmp.get_n<int64_t>(nnzb + 1);
    int64_t* pos = tmp.get_n<int64_t>(nnzb + 1);
    if (nnzb)
      k_item_flags<<<(unsigned)((nnzb + 255) / 256), 256, 0, st>>>(C.rowidx, C.col, nnzb, upper_only ? 1 : 0, flag);
    RT_CUDA_CHECK(cudaGetLastError());
    int64_t n_items = exclusive_scan_i64(flag, pos, nnzb, tmp, st);
    T.n_items = n_items;
    T.item_blk = arena.get_n<int32_t>(n_items);
    if (nnzb) k_item_compact<<<(unsigned)((nnzb + 255) / 256), 256, 0, st>>>(flag, pos, nnzb, T.item_blk);
    int64_t* cnt = tmp.get_n<int64_t>(n_items + 1);
    T.ptr = arena.get_n<int64_t>(n_items + 1);
    if (n_items)
      k_triples<false><<<(unsigned)((n_items + 127) / 128), 128, 0, st>>>(
          T.item_blk, n_items, C.rowidx, C.col, A.rowptr, A.col, A.tmap, a_dag, B.rowptr, B.col, B.tmap, b_dag, cnt,
          nullptr, nullptr);
    RT_CUDA_CHECK(cudaGetLastError());
    T.n_triples = exclusive_scan_i64(cnt, T.ptr, n_items, tmp, st);
    T.ab = arena.get_n<int2>(T.n_triples);
    if (n_items)
      k_triples<true><<<(unsigned)((n_items + 127) / 128), 128, 0, st>>>(
          T.item_blk, n_items, C.rowidx, C.col, A.rowptr, A.col, A.tmap, a_dag, B.rowptr, B.col, B.tmap, b_dag,
          nullptr, T.ptr, T.ab);
    RT_CUDA_CHECK(cudaGetLastError());
    RT_CUDA_CHECK(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    tmp.release_all();
    throw;
  }
  tmp.release_all();
}

// true multiply-adds of a triple list: sum over triples of b_i b_k b_j
__global__ void k_true_macs(const int32_t* __restrict__ item_blk, const int64_t* __restrict__ ptr, int64_t n_items,
                            const int2* __restrict__ ab, const int32_t* __restrict__ c_rowidx,
                            const int32_t* __restrict__ c_col, const int32_t* __restrict__ a_rowidx,
                            const int32_t* __restrict__ a_col, int a_dag, const int32_t* __restrict__ bsize,
                            unsigned long long* __restrict__ out) {
  int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long acc = 0;
  if (it < n_items) {
    int q = item_blk[it];
    int bi = bsize[c_rowidx[q]], bj = bsize[c_col[q]];
    for (int64_t t = ptr[it]; t < ptr[it + 1]; ++t) {
      int a = ab[t].x;
      int k = a_dag ? a_rowidx[a] : a_col[a];
      acc += (unsigned long long)(bi * bsize[k] * bj);
    }
  }
  // warp reduction then one atomic per warp (integer: order-independent)
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

int64_t triple_true_macs(const Triples& T, const Pattern& A, bool a_dag, const Pattern& C, const int32_t* bsize,
                         Arena& arena, cudaStream_t st) {
  if (T.n_items == 0) return 0;
  Arena tmp;
  tmp.alloc = arena.alloc;
  tmp.stream = st;
  unsigned long long h = 0;
  try {
    unsigned long long* d = tmp.get_n<unsigned long long>(1);
    RT_CUDA_CHECK(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    k_true_macs<<<(unsigned)((T.n_items + 255) / 256), 256, 0, st>>>(T.item_blk, T.ptr, T.n_items, T.ab, C.rowidx,
                                                                     C.col, A.rowidx, A.col, a_dag ? 1 : 0, bsize, d);
    RT_CUDA_CHECK(cudaGetLastError());
    RT_CUDA_CHECK(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    RT_CUDA_CHECK(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    tmp.release_all();
    throw;
  }
  tmp.release_all();
  return (int64_t)h;
}

}  // namespace rt
