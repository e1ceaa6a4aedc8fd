// Elementwise and reduction kernels of the step: field update (Sec. II.B),
// identity/Taylor initialisation (eq. matrix_exp), the Crank-Nicolson operands,
// the traces Tr(K S) and Tr(K D_j) (Sec. IV charge, Sec. II.B dipole), the
// unitarity measure of eq. s_unit, and deterministic fixed-order reductions.
#include <cmath>

#include <cstring>

#include "rt_elementwise.cuh"

namespace rt {

// ---------------------------------------------------------------------------
// per-step device state
// ---------------------------------------------------------------------------
__device__ __forceinline__ double field_at(const FieldParams& f, double t) {
  if (f.kind == RT_FIELD_GAUSSIAN) {
    double x = t - f.t0;
    return f.E0 * exp(-(x * x) / (2.0 * f.sigma * f.sigma)) * cos(f.omega * x);
  }
  if (f.kind == RT_FIELD_CONSTANT) return f.E0;
  return 0.0;
}

__global__ void k_begin_step(DevState* s, FieldParams f, double dt, int n_herm) {
  const double t = s->t, r3 = sqrt(3.0);
  s->E[0] = field_at(f, t + 0.5 * dt);
  s->E[1] = field_at(f, t);
  s->E[2] = field_at(f, t + dt);
  s->E[3] = field_at(f, t + (0.5 - r3 / 6.0) * dt);
  s->E[4] = field_at(f, t + (0.5 + r3 / 6.0) * dt);
  for (int i = 0; i < n_herm; ++i) s->herm_bits[i] = 0ull;
}

__global__ void k_end_step(DevState* s, double dt) {
  s->t += dt;
  s->step += 1;
}

void launch_begin_step(DevState* s, const FieldParams& f, double dt, int n_herm, cudaStream_t st) {
  k_begin_step<<<1, 1, 0, st>>>(s, f, dt, n_herm);
  RT_CUDA_CHECK(cudaGetLastError());
}
void launch_end_step(DevState* s, double dt, cudaStream_t st) {
  k_end_step<<<1, 1, 0, st>>>(s, dt);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// H(t+dt/2) = H0 - E D_j
// ---------------------------------------------------------------------------
__global__ void k_field_axpy(const double* __restrict__ H0, const double* __restrict__ D, const DevState* s,
                             int which, double scale, double* __restrict__ Hm, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double E = s ? s->E[which] * scale : scale;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) Hm[i] = H0[i] - E * D[i];
}

void launch_field_axpy(const double* H0, const double* D, const DevState* s, int which, double scale, double* Hm,
                       int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_field_axpy<<<(unsigned)g, 256, 0, st>>>(H0, D, s, which, scale, Hm, n);
  RT_CUDA_CHECK(cudaGetLastError());
}

// M4 exponent (Sec. II.A) on P_U: Om = -i dt/2 (T1 + T2) - (sqrt(3) dt^2/12) [T2, T1]
// with [T2, T1] = C21 - C12 (both cut to P_U); T1, T2 on P_T through u_to_t.
__global__ void k_m4_omega(const double* __restrict__ T1, const double* __restrict__ T2,
                           const int32_t* __restrict__ u_to_t, const double* __restrict__ C21,
                           const double* __restrict__ C12, double dt, double2* __restrict__ Om, int64_t nnzb_u,
                           int NE) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double cc = sqrt(3.0) * dt * dt / 12.0;
  for (; idx < nnzb_u * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int tq = u_to_t ? u_to_t[q] : (int)q;
    double ts = 0.0;
    if (tq >= 0) ts = T1[(int64_t)tq * NE + e] + T2[(int64_t)tq * NE + e];
    Om[idx] = make_double2(-cc * (C21[idx] - C12[idx]), -0.5 * dt * ts);
  }
}

void launch_m4_omega(const double* T1, const double* T2, const int32_t* u_to_t, const double* C21, const double* C12,
                     double dt, double2* Om, int64_t nnzb_u, int B, cudaStream_t st) {
  int64_t n = nnzb_u * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_m4_omega<<<(unsigned)g, 256, 0, st>>>(T1, T2, u_to_t, C21, C12, dt, Om, nnzb_u, B * B);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// U = I + c1 T  (T on P_T mapped into P_U; U complex)
// ---------------------------------------------------------------------------
template <typename CV, typename RV>
__global__ void k_taylor_init(CV* __restrict__ U, int64_t nnzb_u, const int32_t* __restrict__ u_rowidx,
                              const int32_t* __restrict__ u_col, const RV* __restrict__ T,
                              const int32_t* __restrict__ u_to_t, int B, int urs, double c1, int c1_imag,
                              int ident) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb_u * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    double re = (ident && u_rowidx[q] == u_col[q] && r == c) ? 1.0 : 0.0;
    double im = 0.0;
    int tq = u_to_t ? u_to_t[q] : (int)q;
    if (tq >= 0) {
      double tv = (double)T[(int64_t)tq * NE + e];
      if (c1_imag) im += c1 * tv;
      else re += c1 * tv;
    }
    CV v;
    v.x = (decltype(v.x))re;
    v.y = (decltype(v.y))im;
    U[q * (int64_t)B * urs + r * urs + c] = v;
  }
}

// U (FP64, dense blocks) = ident*I + c1 T, or the FP32 difference dU = c1 T
// in the FP32 block layout (row stride rs32(B)); T is FP64 with dense blocks.
void launch_taylor_init(void* U, bool fp32, int64_t nnzb_u, const int32_t* u_rowidx, const int32_t* u_col,
                        const void* T, bool t_fp32, const int32_t* u_to_t, int B, double c1, int c1_imag, int ident,
                        cudaStream_t st) {
  int64_t n = nnzb_u * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (t_fp32) throw Error{RT_EINTERNAL, "taylor init takes an FP64 T"};
  if (!fp32)
    k_taylor_init<double2, double><<<(unsigned)g, 256, 0, st>>>((double2*)U, nnzb_u, u_rowidx, u_col,
                                                                (const double*)T, u_to_t, B, B, c1, c1_imag, ident);
  else
    k_taylor_init<float2, double><<<(unsigned)g, 256, 0, st>>>((float2*)U, nnzb_u, u_rowidx, u_col,
                                                               (const double*)T, u_to_t, B, rs32(B), c1, c1_imag,
                                                               ident);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// identity * scale on a pattern (real or complex FP64)
// ---------------------------------------------------------------------------
__global__ void k_identity(double* __restrict__ X, int cplx, int64_t nnzb, const int32_t* __restrict__ rowidx,
                           const int32_t* __restrict__ col, int B, double scale) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    double v = (rowidx[q] == col[q] && r == c) ? scale : 0.0;
    if (cplx) {
      X[2 * idx] = v;
      X[2 * idx + 1] = 0.0;
    } else {
      X[idx] = v;
    }
  }
}

void launch_identity(double* X, bool cplx, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B,
                     double scale, cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_identity<<<(unsigned)g, 256, 0, st>>>(X, cplx ? 1 : 0, nnzb, rowidx, col, B, scale);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// gather a matrix onto another pattern through a block map (cut / zero-extend)
// mode 0: real -> real, 1: real -> complex, 2: complex -> complex
// ---------------------------------------------------------------------------
__global__ void k_restrict(const double* __restrict__ src, double* __restrict__ dst, const int32_t* __restrict__ map,
                           int64_t nnzb_dst, int NE, int mode) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; idx < nnzb_dst * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int sq = map[q];
    if (mode == 0) {
      dst[idx] = sq >= 0 ? src[(int64_t)sq * NE + e] : 0.0;
    } else if (mode == 1) {
      dst[2 * idx] = sq >= 0 ? src[(int64_t)sq * NE + e] : 0.0;
      dst[2 * idx + 1] = 0.0;
    } else {
      dst[2 * idx] = sq >= 0 ? src[2 * ((int64_t)sq * NE + e)] : 0.0;
      dst[2 * idx + 1] = sq >= 0 ? src[2 * ((int64_t)sq * NE + e) + 1] : 0.0;
    }
  }
}

void launch_restrict(const double* src, double* dst, const int32_t* map, int64_t nnzb_dst, int B, int mode,
                     cudaStream_t st) {
  int64_t n = nnzb_dst * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_restrict<<<(unsigned)g, 256, 0, st>>>(src, dst, map, nnzb_dst, B * B, mode);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// CN operands on P_A: A = S + i c H, Bm = S - i c H  (S, H gathered by maps)
// ---------------------------------------------------------------------------
__global__ void k_cn_operands(const double* __restrict__ S, const int32_t* __restrict__ a_to_s,
                              const double* __restrict__ H, const int32_t* __restrict__ a_to_h, double c,
                              double2* __restrict__ A, double2* __restrict__ Bm, int64_t nnzb_a, int NE) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; idx < nnzb_a * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int sq = a_to_s[q], hq = a_to_h[q];
    double s = sq >= 0 ? S[(int64_t)sq * NE + e] : 0.0;
    double h = hq >= 0 ? H[(int64_t)hq * NE + e] : 0.0;
    A[idx] = make_double2(s, c * h);
    Bm[idx] = make_double2(s, -c * h);
  }
}

void launch_cn_operands(const double* S, const int32_t* a_to_s, const double* H, const int32_t* a_to_h, double c,
                        double2* A, double2* Bm, int64_t nnzb_a, int B, cudaStream_t st) {
  int64_t n = nnzb_a * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_cn_operands<<<(unsigned)g, 256, 0, st>>>(S, a_to_s, H, a_to_h, c, A, Bm, nnzb_a, B * B);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
constexpr int RED_T = 256;
constexpr int RED_MAXB = 1024;

// sum of vals[0..n) in a fixed order: per-block strided partial sums, then one
// block adds the partials in index order.
__global__ void k_sum_partials(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double s[RED_T];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RED_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_T) acc += v[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int off = RED_T / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_sum_final(const double* __restrict__ part, int nb, double scale_sqrt_div, double* out,
                            double* out2) {
  __shared__ double s[RED_T];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += RED_T) acc += part[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int off = RED_T / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) s[threadIdx.x] += s[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r = s[0];
    if (scale_sqrt_div > 0.0) r = sqrt(r) / scale_sqrt_div;
    *out = r;
    if (out2) *out2 = r;
  }
}

int reduce_blocks(int64_t n) {
  int64_t b = (n + RED_T - 1) / RED_T;
  if (b < 1) b = 1;
  if (b > RED_MAXB) b = RED_MAXB;
  return (int)b;
}

void launch_sum(const double* v, int64_t n, double* part, double sqrt_div, double* out, double* out2, cudaStream_t st) {
  int nb = reduce_blocks(n);
  k_sum_partials<<<nb, RED_T, 0, st>>>(v, n, part);
  k_sum_final<<<1, RED_T, 0, st>>>(part, nb, sqrt_div, out, out2);
  RT_CUDA_CHECK(cudaGetLastError());
}

// Tr(K X) for X in {S, Dx, Dy, Dz}.  K is hermitian (upper blocks mirrored,
// diagonal blocks symmetrised) and every X is real symmetric, so
//   Tr(K X) = sum_{i<j} 2 sum_ab Re K_ij[a,b] X_ji[b,a] + sum_i sum_ab Re K_ii[a,b] X_ii[b,a]
// and Im Tr(K X) = 0 exactly; only the upper blocks are read.  X_ji comes
// through kx_map (block (j,i) of X, or -1).  One warp per block (coalesced
// reads of K), fixed block-to-warp assignment and fixed-order reductions: the
// result does not depend on scheduling.
// One CTA's share (block index blk of nblk) of the trace sums of one K; its
// 8 partials go to part[blk * 8 ..].
__device__ __forceinline__ void traces_cta(const double2* __restrict__ K, int64_t nnzb,
                                           const int32_t* __restrict__ rowidx, const int32_t* __restrict__ col,
                                           const int32_t* __restrict__ bsize, int B, const double* __restrict__ S,
                                           const int32_t* __restrict__ ks_map, const double* __restrict__ Dx,
                                           const double* __restrict__ Dy, const double* __restrict__ Dz,
                                           const int32_t* __restrict__ kd_map, double* __restrict__ part, int blk,
                                           int nblk) {
  __shared__ double s[4][RED_T / 32];
  double acc[4] = {0, 0, 0, 0};
  const int NE = B * B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blk * (RED_T / 32) + warp;
  const int64_t nw = (int64_t)nblk * (RED_T / 32);
  for (int64_t q = gw; q < nnzb; q += nw) {
    int i = rowidx[q], j = col[q];
    if (j < i) continue;
    const double w = (i == j) ? 1.0 : 2.0;
    int bi = bsize[i], bj = bsize[j];
    int sq = ks_map[q], dq = kd_map[q];
    const double2* k = K + q * NE;
    for (int e = lane; e < bi * bj; e += 32) {
      int a = e / bj, b = e - a * bj;
      double kr = w * k[a * B + b].x;
      int te = b * B + a;  // X_ji[b][a]
      if (sq >= 0) acc[0] += kr * S[(int64_t)sq * NE + te];
      if (dq >= 0) {
        acc[1] += kr * Dx[(int64_t)dq * NE + te];
        acc[2] += kr * Dy[(int64_t)dq * NE + te];
        acc[3] += kr * Dz[(int64_t)dq * NE + te];
      }
    }
  }
  for (int c = 0; c < 4; ++c)
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], off);
  if (lane == 0)
    for (int c = 0; c < 4; ++c) s[c][warp] = acc[c];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; ++c) {
      double t = 0.0;
      for (int w = 0; w < RED_T / 32; ++w) t += s[c][w];
      part[blk * 8 + 2 * c] = t;
      part[blk * 8 + 2 * c + 1] = 0.0;  // Im Tr(K X) = 0 for hermitian K, symmetric X
    }
}

__global__ void k_traces(const double2* __restrict__ K, int64_t nnzb, const int32_t* __restrict__ rowidx,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ bsize, int B,
                         const double* __restrict__ S, const int32_t* __restrict__ ks_map,
                         const double* __restrict__ Dx, const double* __restrict__ Dy, const double* __restrict__ Dz,
                         const int32_t* __restrict__ kd_map, double* __restrict__ part) {
  traces_cta(K, nnzb, rowidx, col, bsize, B, S, ks_map, Dx, Dy, Dz, kd_map, part, blockIdx.x, gridDim.x);
}

// The same for every (system, kick) pair of a table: pair blockIdx.y, its
// partials at part[pair * gridDim.x * 8 ..].
__global__ void k_traces_grouped(const TracePair* __restrict__ tab, double* __restrict__ part) {
  const TracePair& t = tab[blockIdx.y];
  traces_cta(t.K, t.nnzb, t.rowidx, t.col, t.bsize, t.B, t.S, t.ks_map, t.Dx, t.Dy, t.Dz, t.kd_map,
             part + (int64_t)blockIdx.y * gridDim.x * 8, blockIdx.x, gridDim.x);
}

// Sums the trace partials in fixed order and writes one observables record.
__device__ __forceinline__ void traces_final_cta(const double* __restrict__ part, int nb, const DevState* st,
                                                 int herm_slot, double* __restrict__ ring, int capacity, int n_slots,
                                                 int slot_index, const double* __restrict__ ref,
                                                 double* __restrict__ out) {
  __shared__ double s[8][RED_T];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nb; i += RED_T)
    for (int c = 0; c < 8; ++c) acc[c] += part[i * 8 + c];
  for (int c = 0; c < 8; ++c) s[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int off = RED_T / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int c = 0; c < 8; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0 && ref)  // incremental form: traces of K_ref + dK
    for (int c = 0; c < 8; ++c) s[c][0] += ref[c];
  if (threadIdx.x == 0 && out) {  // plain output (reference traces)
    for (int c = 0; c < 8; ++c) out[c] = s[c][0];
    return;
  }
  if (threadIdx.x == 0) {
    int64_t step = st->step - 1;  // runs after the step counter advanced
    int64_t r = step % capacity;
    double* rec = ring + (r * n_slots + slot_index) * RT_NOBS;
    rec[RT_OBS_T] = st->t;
    // Tr(KX) = sum K X^T: real part from K.re, imaginary from K.im (X real)
    rec[RT_OBS_TRKS_RE] = s[0][0];
    rec[RT_OBS_TRKS_IM] = s[1][0];
    rec[RT_OBS_TRKDX_RE] = s[2][0];
    rec[RT_OBS_TRKDX_IM] = s[3][0];
    rec[RT_OBS_TRKDY_RE] = s[4][0];
    rec[RT_OBS_TRKDY_IM] = s[5][0];
    rec[RT_OBS_TRKDZ_RE] = s[6][0];
    rec[RT_OBS_TRKDZ_IM] = s[7][0];
    rec[RT_OBS_HERM] = __longlong_as_double((long long)st->herm_bits[herm_slot]);
    rec[RT_OBS_HOT_ITERS] = st->hot_iters;
    rec[RT_OBS_HOT_RESID] = st->hot_resid;
  }
}

__global__ void k_traces_final(const double* __restrict__ part, int nb, const DevState* st, int herm_slot,
                               double* __restrict__ ring, int capacity, int n_slots, int slot_index,
                               const double* __restrict__ ref, double* __restrict__ out) {
  traces_final_cta(part, nb, st, herm_slot, ring, capacity, n_slots, slot_index, ref, out);
}

// One record per pair of the table (pair blockIdx.x)
__global__ void k_traces_final_grouped(const TracePair* __restrict__ tab, const double* __restrict__ part, int nb,
                                       const DevState* st, double* __restrict__ ring, int capacity, int n_slots) {
  const TracePair& t = tab[blockIdx.x];
  traces_final_cta(part + (int64_t)blockIdx.x * nb * 8, nb, st, t.herm_slot, ring, capacity, n_slots, t.slot_index,
                   t.ref, nullptr);
}

void launch_traces(const double2* K, int64_t nnzb, const int32_t* rowidx, const int32_t* col, const int32_t* bsize,
                   int B, const double* S, const int32_t* ks_map, const double* Dx, const double* Dy,
                   const double* Dz, const int32_t* kd_map, double* part, const DevState* st, int herm_slot,
                   double* ring, int capacity, int n_slots, int slot_index, cudaStream_t s, const double* ref,
                   double* out) {
  int nb = reduce_blocks(nnzb);
  k_traces<<<nb, RED_T, 0, s>>>(K, nnzb, rowidx, col, bsize, B, S, ks_map, Dx, Dy, Dz, kd_map, part);
  k_traces_final<<<1, RED_T, 0, s>>>(part, nb, st, herm_slot, ring, capacity, n_slots, slot_index, ref, out);
  RT_CUDA_CHECK(cudaGetLastError());
}

void launch_traces_grouped(const TracePair* tab, int n_pairs, int nb, double* part, const DevState* st, double* ring,
                           int capacity, int n_slots, cudaStream_t s) {
  if (n_pairs == 0) return;
  RT_REQUIRE(nb >= 1 && nb <= RED_MAXB && n_pairs < 65536, RT_EINTERNAL, "grouped traces: bad launch shape");
  k_traces_grouped<<<dim3((unsigned)nb, (unsigned)n_pairs), RED_T, 0, s>>>(tab, part);
  k_traces_final_grouped<<<(unsigned)n_pairs, RED_T, 0, s>>>(tab, part, nb, st, ring, capacity, n_slots);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// unitarity: |E - Ref| over the true entries of P_U (max and sum)
// Ref = S gathered on P_U (metric) or the identity.
// ---------------------------------------------------------------------------
__global__ void k_unit_dev(const double2* __restrict__ E, int64_t nnzb, const int32_t* __restrict__ rowidx,
                           const int32_t* __restrict__ col, const int32_t* __restrict__ bsize, int B,
                           const double* __restrict__ S, const int32_t* __restrict__ us_map,
                           double* __restrict__ part_max, double* __restrict__ part_sum) {
  __shared__ double smax[RED_T], ssum[RED_T];
  double mx = 0.0, sm = 0.0;
  const int NE = B * B;
  for (int64_t q = (int64_t)blockIdx.x * RED_T + threadIdx.x; q < nnzb; q += (int64_t)gridDim.x * RED_T) {
    int i = rowidx[q], j = col[q];
    int bi = bsize[i], bj = bsize[j];
    int sq = us_map ? us_map[q] : -1;
    for (int a = 0; a < bi; ++a)
      for (int b = 0; b < bj; ++b) {
        double2 e = E[q * NE + a * B + b];
        double ref;
        if (us_map) ref = sq >= 0 ? S[(int64_t)sq * NE + a * B + b] : 0.0;
        else ref = (i == j && a == b) ? 1.0 : 0.0;
        double dr = e.x - ref, di = e.y;
        double d = sqrt(dr * dr + di * di);
        mx = fmax(mx, d);
        sm += d;
      }
  }
  smax[threadIdx.x] = mx;
  ssum[threadIdx.x] = sm;
  __syncthreads();
  for (int off = RED_T / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + off]);
      ssum[threadIdx.x] += ssum[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part_max[blockIdx.x] = smax[0];
    part_sum[blockIdx.x] = ssum[0];
  }
}

int launch_unitarity_dev(const double2* E, int64_t nnzb, const int32_t* rowidx, const int32_t* col,
                         const int32_t* bsize, int B, const double* S, const int32_t* us_map, double* part_max,
                         double* part_sum, cudaStream_t st) {
  int nb = reduce_blocks(nnzb);
  k_unit_dev<<<nb, RED_T, 0, st>>>(E, nnzb, rowidx, col, bsize, B, S, us_map, part_max, part_sum);
  RT_CUDA_CHECK(cudaGetLastError());
  return nb;
}

// ---------------------------------------------------------------------------
// max_i sum_j |S_ij| over true entries (Gershgorin bound of Hotelling's X0)
// ---------------------------------------------------------------------------
__global__ void k_row_abs_sums(const double* __restrict__ S, const int32_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ bsize, int B, int n_atoms,
                               double* __restrict__ rows) {
  int i = blockIdx.x;
  if (i >= n_atoms) return;
  int bi = bsize[i];
  for (int a = threadIdx.x; a < bi; a += blockDim.x) {
    double acc = 0.0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      int j = col[q];
      for (int b = 0; b < bsize[j]; ++b) acc += fabs(S[(int64_t)q * B * B + a * B + b]);
    }
    rows[(int64_t)i * B + a] = acc;
  }
}

__global__ void k_max_final(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double s[RED_T];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += RED_T) m = fmax(m, v[i]);
  s[threadIdx.x] = m;
  __syncthreads();
  for (int off = RED_T / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

void launch_inf_norm(const double* S, const int32_t* rowptr, const int32_t* col, const int32_t* bsize, int B,
                     int n_atoms, double* rows_tmp, double* out, cudaStream_t st) {
  RT_CUDA_CHECK(cudaMemsetAsync(rows_tmp, 0, sizeof(double) * (size_t)n_atoms * B, st));
  k_row_abs_sums<<<n_atoms, 32, 0, st>>>(S, rowptr, col, bsize, B, n_atoms, rows_tmp);
  k_max_final<<<1, RED_T, 0, st>>>(rows_tmp, (int64_t)n_atoms * B, out);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Chebyshev step of the Fermi-operator expansion (real FP64, on P_K):
//   xy = (TY - a Y)/w;  Ynew = first ? xy : 2 xy - Yprev;  K += c Ynew
// ---------------------------------------------------------------------------
__global__ void k_cheb_step(const double* __restrict__ TY, const double* __restrict__ Y, const double* __restrict__ Yp,
                            double* __restrict__ Yn, double* __restrict__ Kacc, double a, double w, double c, int first,
                            int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double xy = (TY[i] - a * Y[i]) / w;
    double yn = first ? xy : 2.0 * xy - Yp[i];
    Yn[i] = yn;
    Kacc[i] = Kacc[i] + c * yn;
  }
}

void launch_cheb_step(const double* TY, const double* Y, const double* Yp, double* Yn, double* Kacc, double a,
                      double w, double c, int first, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_cheb_step<<<(unsigned)g, 256, 0, st>>>(TY, Y, Yp, Yn, Kacc, a, w, c, first, n);
  RT_CUDA_CHECK(cudaGetLastError());
}

__global__ void k_scale(double* __restrict__ v, double c, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] = c * v[i];
}

void launch_scale(double* v, double c, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_scale<<<(unsigned)g, 256, 0, st>>>(v, c, n);
  RT_CUDA_CHECK(cudaGetLastError());
}

// K0 <- (K0 + K0^T)/2 as complex (imaginary zero), padded entries zero
__global__ void k_symmetrise_to_complex(const double* __restrict__ Kr, double2* __restrict__ K, int64_t nnzb,
                                        const int32_t* __restrict__ rowidx, const int32_t* __restrict__ col,
                                        const int32_t* __restrict__ tmap, const int32_t* __restrict__ bsize, int B) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    int i = rowidx[q], j = col[q];
    double v = 0.0;
    if (r < bsize[i] && c < bsize[j]) v = 0.5 * (Kr[idx] + Kr[(int64_t)tmap[q] * NE + c * B + r]);
    K[idx] = make_double2(v, 0.0);
  }
}

void launch_symmetrise_to_complex(const double* Kr, double2* K, int64_t nnzb, const int32_t* rowidx,
                                  const int32_t* col, const int32_t* tmap, const int32_t* bsize, int B,
                                  cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_symmetrise_to_complex<<<(unsigned)g, 256, 0, st>>>(Kr, K, nnzb, rowidx, col, tmap, bsize, B);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// precision conversions and the delta-form operand W = K + M (FP32)
// ---------------------------------------------------------------------------
// FP64 dense blocks -> FP32 blocks with row stride rs (ncomp = 1 real, 2 complex)
__global__ void k_d2f_pad(const double* __restrict__ a, float* __restrict__ b, int64_t nnzb, int B, int rs,
                          int ncomp) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    int64_t o = q * (int64_t)B * rs + r * rs + c;
    for (int k = 0; k < ncomp; ++k) b[ncomp * o + k] = (float)a[ncomp * idx + k];
  }
}

void launch_d2f_pad(const double* a, float* b, int64_t nnzb, int B, bool cplx, cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_d2f_pad<<<(unsigned)g, 256, 0, st>>>(a, b, nnzb, B, rs32(B), cplx ? 2 : 1);
  RT_CUDA_CHECK(cudaGetLastError());
}

// dUH[q] = conj(dU[q])^T (FP32 complex, same block index, FP32 block layout)
__global__ void k_dagger32(const float2* __restrict__ dU, float2* __restrict__ dUH, int64_t nnzb, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    float2 v = dU[q * (int64_t)B * rs + c * rs + r];
    dUH[q * (int64_t)B * rs + r * rs + c] = make_float2(v.x, -v.y);
  }
}

void launch_dagger32(const float2* dU, float2* dUH, int64_t nnzb, int B, cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_dagger32<<<(unsigned)g, 256, 0, st>>>(dU, dUH, nnzb, B, rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

// W[q] = (float)K[mk[q]] + M[q] on P_M (complex; K dense FP64 blocks, M and
// W in the FP32 block layout)
__global__ void k_delta_w(const double2* __restrict__ K, const int32_t* __restrict__ m_to_k,
                          const float2* __restrict__ Mf, float2* __restrict__ Wf, int64_t nnzb_m, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb_m * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    int64_t o = q * (int64_t)B * rs + r * rs + c;
    int kq = m_to_k ? m_to_k[q] : (int)q;
    float2 m = Mf[o];
    if (kq >= 0) {
      double2 k = K[(int64_t)kq * NE + e];
      m.x = (float)((double)m.x + k.x);
      m.y = (float)((double)m.y + k.y);
    }
    Wf[o] = m;
  }
}

void launch_delta_w(const double2* K, const int32_t* m_to_k, const float2* Mf, float2* Wf, int64_t nnzb_m, int B,
                    cudaStream_t st) {
  int64_t n = nnzb_m * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_delta_w<<<(unsigned)g, 256, 0, st>>>(K, m_to_k, Mf, Wf, nnzb_m, B, rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

__global__ void k_set_hot(DevState* s, const double* resid, int iters) {
  s->hot_resid = *resid;
  s->hot_iters = iters;
}

void launch_set_hot(DevState* s, const double* resid, int iters, cudaStream_t st) {
  k_set_hot<<<1, 1, 0, st>>>(s, resid, iters);
  RT_CUDA_CHECK(cudaGetLastError());
}

// dU = U - I in FP32 (CN delta form)
__global__ void k_u_minus_i_f32(const double2* __restrict__ U, float2* __restrict__ dU, int64_t nnzb,
                                const int32_t* __restrict__ rowidx, const int32_t* __restrict__ col, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    double2 u = U[idx];
    double d = (rowidx[q] == col[q] && r == c) ? 1.0 : 0.0;
    dU[q * (int64_t)B * rs + r * rs + c] = make_float2((float)(u.x - d), (float)u.y);
  }
}

void launch_u_minus_i_f32(const double2* U, float2* dU, int64_t nnzb, const int32_t* rowidx, const int32_t* col,
                          int B, cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_u_minus_i_f32<<<(unsigned)g, 256, 0, st>>>(U, dU, nnzb, rowidx, col, B, rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

// U = I + dU (FP32 difference promoted to FP64), for diagnostics of the mixed path
__global__ void k_u_from_delta(const float2* __restrict__ dU, double2* __restrict__ U, int64_t nnzb,
                               const int32_t* __restrict__ rowidx, const int32_t* __restrict__ col, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int r = e / B, c = e - r * B;
    float2 d = dU[q * (int64_t)B * rs + r * rs + c];
    double one = (rowidx[q] == col[q] && r == c) ? 1.0 : 0.0;
    U[idx] = make_double2(one + (double)d.x, (double)d.y);
  }
}

void launch_u_from_delta(const float2* dU, double2* U, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B,
                         cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_u_from_delta<<<(unsigned)g, 256, 0, st>>>(dU, U, nnzb, rowidx, col, B, rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

// Stochastic rounding to FP32 (reference-split form).  A fixed FP32 rounding
// of U - I is the same perturbation of the propagator at every step, and its
// effect on the induced dipole grows linearly with the step count; rounding
// each element to one of its two neighbouring floats at random, with the
// probabilities that make the result unbiased, turns that drift into a random
// walk.  The uniform bits come from a counter: the SplitMix64 output function
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014) of a key made of the step number and the element index, so a
// run is reproducible and a replayed step graph draws fresh numbers.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// x (FP64) stochastically rounded to FP32 with 29 random bits r: adding r to
// the 29 mantissa bits of x below FP32 precision and cutting them off leaves
// the float just below |x| or, if the addition carried, the next one up; the
// carry happens with probability equal to the fraction of a float ulp by which
// |x| exceeds the lower float, so E[result] = x (the add-and-truncate form of
// stochastic rounding, Croci et al., "Stochastic rounding: implementation,
// error analysis and applications", R. Soc. Open Sci. 9, 2022).  The sign bit
// is untouched (the magnitude is rounded), a carry into the exponent gives the
// next binade, and the truncated double has 23 mantissa bits, so the final
// conversion is exact for values in the normal FP32 range.
__device__ __forceinline__ float round_sr(double x, uint32_t r29) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  b = (b + (r29 & 0x1FFFFFFFu)) & ~0x1FFFFFFFull;
  return (float)__longlong_as_double((long long)b);
}

__device__ __forceinline__ uint64_t sr_bits(int64_t step, int64_t idx) {
  return splitmix64(((uint64_t)step << 34) ^ (uint64_t)idx);
}

// Writes one block's FP32 dU (from the FP64 values in v, 32 lanes of a warp
// over the B*B elements, row-major; rounded to nearest or stochastically) and
// its conjugate transpose dUH through the warp's shared tile, so that both
// stores run along rows.
constexpr int POLY_WARPS = 8;
__device__ __forceinline__ void store_du_block(float2* __restrict__ tile, double2 v, int e, int B, int rs, int64_t q,
                                              bool diag, int stochastic, int64_t step, int64_t idx,
                                              float2* __restrict__ dU) {
  const int r = e / B, c = e - r * B;
  const double d = (diag && r == c) ? 1.0 : 0.0;
  float2 f;
  if (stochastic) {
    const uint64_t z = sr_bits(step, idx);
    f = make_float2(round_sr(v.x - d, (uint32_t)z), round_sr(v.y, (uint32_t)(z >> 32)));
  } else {
    f = make_float2((float)(v.x - d), (float)v.y);
  }
  if (dU) dU[q * (int64_t)B * rs + r * rs + c] = f;
  tile[e] = f;
}

// The block in the tile written column-planar (13-function blocks, 416
// floats: for each column m the real parts of rows 0..15, then the
// imaginary parts; rows 13..15 zero), the A layout of the packed FP32
// product kernel; coalesced stores.
__device__ __forceinline__ void store_planar_block(const float2* __restrict__ tile, int lane, int64_t q,
                                                   float2* __restrict__ dU) {
  constexpr int B = 13, RS = 16;
  float* __restrict__ D = reinterpret_cast<float*>(dU) + q * (int64_t)(2 * B * RS);
  for (int idx = lane; idx < 2 * B * RS; idx += 32) {
    const int m = idx / (2 * RS), w = idx % (2 * RS), r = w % RS;
    float v = 0.f;
    if (r < B) {
      const float2 t = tile[r * B + m];
      v = w >= RS ? t.y : t.x;
    }
    D[idx] = v;
  }
}

__device__ __forceinline__ void store_dagger_block(const float2* __restrict__ tile, int lane, int B, int rs, int64_t q,
                                                  float2* __restrict__ dUH) {
  const int NE = B * B;
  for (int e = lane; e < NE; e += 32) {
    const int r = e / B, c = e - r * B;
    const float2 t = tile[c * B + r];
    dUH[q * (int64_t)B * rs + r * rs + c] = make_float2(t.x, -t.y);
  }
}

// dU = U - I stochastically rounded to FP32 (FP32 block layout) and its
// per-block conjugate transpose dUH, from a constant FP64 U; one warp per
// block, draws keyed on the step number held in the device state.
__global__ void __launch_bounds__(POLY_WARPS * 32) k_round_u_sr(const double2* __restrict__ U, float2* __restrict__ dU,
                                                                float2* __restrict__ dUH, int64_t nnzb,
                                                                const int32_t* __restrict__ rowidx,
                                                                const int32_t* __restrict__ col, int B, int rs,
                                                                const DevState* __restrict__ s, int planar) {
  __shared__ float2 tiles[POLY_WARPS][13 * 13];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t step = s->step;
  const int NE = B * B;
  for (int64_t q = (int64_t)blockIdx.x * POLY_WARPS + warp; q < nnzb; q += (int64_t)gridDim.x * POLY_WARPS) {
    const bool diag = rowidx[q] == col[q];
    for (int e = lane; e < NE; e += 32) {
      const int64_t idx = q * NE + e;
      store_du_block(tiles[warp], U[idx], e, B, rs, q, diag, 1, step, idx, planar ? nullptr : dU);
    }
    __syncwarp();
    if (planar) store_planar_block(tiles[warp], lane, q, dU);
    if (dUH) store_dagger_block(tiles[warp], lane, B, rs, q, dUH);
    __syncwarp();
  }
}

static int64_t poly_grid(int64_t nnzb) {
  int64_t g = (nnzb + POLY_WARPS - 1) / POLY_WARPS;
  return g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g);
}

void launch_round_u_sr(const double2* U, float2* dU, float2* dUH, int64_t nnzb, const int32_t* rowidx,
                       const int32_t* col, int B, const DevState* s, cudaStream_t st, bool planar) {
  if (nnzb == 0) return;
  RT_REQUIRE(B <= 13, RT_EINTERNAL, "block size above 13");
  RT_REQUIRE(!planar || B == 13, RT_EINTERNAL, "column-planar blocks are 13-function blocks");
  k_round_u_sr<<<(unsigned)poly_grid(nnzb), POLY_WARPS * 32, 0, st>>>(U, dU, dUH, nnzb, rowidx, col, B, rs32(B), s,
                                                                      planar ? 1 : 0);
  RT_CUDA_CHECK(cudaGetLastError());
}

// R = sum_{p<=deg} E^p C_p (Horner, FP64) on the upper blocks (col >= row) of
// a pattern, E = s->E[which]; the lower blocks of R are not written.
__global__ void __launch_bounds__(POLY_WARPS * 32) k_poly_upper(PolyTerms C, int deg, const DevState* __restrict__ s,
                                                                int which, double2* __restrict__ R, int64_t nnzb,
                                                                const int32_t* __restrict__ rowidx,
                                                                const int32_t* __restrict__ col, int NE) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double E = s->E[which];
  for (int64_t q = (int64_t)blockIdx.x * POLY_WARPS + warp; q < nnzb; q += (int64_t)gridDim.x * POLY_WARPS) {
    if (col[q] < rowidx[q]) continue;  // whole warp: lower blocks are not needed
    for (int e = lane; e < NE; e += 32) {
      const int64_t idx = q * NE + e;
      double2 v = C.v[deg][idx];
      for (int p = deg - 1; p >= 0; --p) {
        const double2 cp = C.v[p][idx];
        v = make_double2(fma(v.x, E, cp.x), fma(v.y, E, cp.y));
      }
      R[idx] = v;
    }
  }
}

void launch_poly_upper(const PolyTerms& C, int deg, const DevState* s, int which, double2* R, int64_t nnzb,
                       const int32_t* rowidx, const int32_t* col, int B, cudaStream_t st) {
  RT_REQUIRE(deg >= 0 && deg < RT_MAX_POLY, RT_EINTERNAL, "polynomial degree out of range");
  if (nnzb == 0) return;
  k_poly_upper<<<(unsigned)poly_grid(nnzb), POLY_WARPS * 32, 0, st>>>(C, deg, s, which, R, nnzb, rowidx, col, B * B);
  RT_CUDA_CHECK(cudaGetLastError());
}

// b = (float)a, complex, n elements (round to nearest)
__global__ void k_z2c(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

void launch_z2c(const double2* a, float2* b, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_z2c<<<(unsigned)g, 256, 0, st>>>(a, b, n);
  RT_CUDA_CHECK(cudaGetLastError());
}

// z = x + a*y (complex FP64 vectors of n elements)
__global__ void k_zaxpy(double2* __restrict__ z, const double2* __restrict__ x, const double2* __restrict__ y, double a,
                        int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 xv = x[i], yv = y[i];
    z[i] = make_double2(xv.x + a * yv.x, xv.y + a * yv.y);
  }
}

void launch_zaxpy(double2* z, const double2* x, const double2* y, double a, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_zaxpy<<<(unsigned)g, 256, 0, st>>>(z, x, y, a, n);
  RT_CUDA_CHECK(cudaGetLastError());
}

// z = x + a y (FP32 complex, element by element; FP32 block layout with its
// zero padding columns, which stay zero)
__global__ void k_axpy32(float2* __restrict__ z, const float2* __restrict__ x, const float2* __restrict__ y, float a,
                         int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 xv = x[i], yv = y[i];
    z[i] = make_float2(fmaf(a, yv.x, xv.x), fmaf(a, yv.y, xv.y));
  }
}

void launch_axpy32(float2* z, const float2* x, const float2* y, float a, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_axpy32<<<(unsigned)g, 256, 0, st>>>(z, x, y, a, n);
  RT_CUDA_CHECK(cudaGetLastError());
}

// Mixed-mode M4 exponent on P_U in the FP32 block layout:
// Om = -i dt/2 (T1 + T2) - (sqrt(3) dt^2/12) (C21 - C12), the field part from
// the FP64 T1, T2 on P_T (through u_to_t), the commutator from the FP32
// products C21 = cut(T2 T1), C12 = cut(T1 T2); dU = Om as the first term of
// exp(Om) - I (zero when the series has only its identity term).
__global__ void k_m4_omega32(const double* __restrict__ T1, const double* __restrict__ T2,
                             const int32_t* __restrict__ u_to_t, const float* __restrict__ C21,
                             const float* __restrict__ C12, double dt, float2* __restrict__ Om,
                             float2* __restrict__ dU, int first_term, int64_t nnzb_u, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int NE = B * B;
  const double cc = sqrt(3.0) * dt * dt / 12.0;
  for (; idx < nnzb_u * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx / NE;
    const int e = (int)(idx - q * NE);
    const int r = e / B, c = e - r * B;
    const int tq = u_to_t ? u_to_t[q] : (int)q;
    double ts = 0.0;
    if (tq >= 0) ts = T1[(int64_t)tq * NE + e] + T2[(int64_t)tq * NE + e];
    const int64_t pidx = q * (int64_t)B * rs + r * rs + c;
    const float2 om = make_float2((float)(-cc * ((double)C21[pidx] - (double)C12[pidx])), (float)(-0.5 * dt * ts));
    Om[pidx] = om;
    dU[pidx] = first_term ? om : make_float2(0.f, 0.f);
  }
}

void launch_m4_omega32(const double* T1, const double* T2, const int32_t* u_to_t, const float* C21, const float* C12,
                       double dt, float2* Om, float2* dU, bool first_term, int64_t nnzb_u, int B, cudaStream_t st) {
  int64_t n = nnzb_u * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_m4_omega32<<<(unsigned)g, 256, 0, st>>>(T1, T2, u_to_t, C21, C12, dt, Om, dU, first_term ? 1 : 0, nnzb_u, B,
                                            rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// field polynomial of the EM propagator
// ---------------------------------------------------------------------------
__global__ void k_acc_real(double2* __restrict__ V, const double* __restrict__ Q, const int32_t* __restrict__ map,
                           int64_t nnzb_v, int NE, double coef, int imag) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; idx < nnzb_v * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx / NE;
    int e = (int)(idx - q * NE);
    int sq = map ? map[q] : (int)q;
    if (sq < 0) continue;
    double v = coef * Q[(int64_t)sq * NE + e];
    if (imag) V[idx].y += v;
    else V[idx].x += v;
  }
}

void launch_acc_real(double2* V, const double* Q, const int32_t* map, int64_t nnzb_v, int B, double coef, int imag,
                     cudaStream_t st) {
  int64_t n = nnzb_v * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_acc_real<<<(unsigned)g, 256, 0, st>>>(V, Q, map, nnzb_v, B * B, coef, imag);
  RT_CUDA_CHECK(cudaGetLastError());
}

// U = sum_m E^m V_m by Horner in FP64, one warp per block (coalesced reads of
// the V_m); FP64 U and/or FP32 dU = U - I with its block dagger dUH.
__global__ void __launch_bounds__(POLY_WARPS * 32) k_field_poly(PolyTerms V, int deg, const DevState* __restrict__ s,
                                                                int which, double2* __restrict__ U,
                                                                float2* __restrict__ dU, float2* __restrict__ dUH,
                                                                int64_t nnzb, const int32_t* __restrict__ rowidx,
                                                                const int32_t* __restrict__ col, int B, int rs,
                                                                int stochastic, int planar, PolyTerms32 T,
                                                                int tail) {
  __shared__ float2 tiles[POLY_WARPS][13 * 13];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double E = s->E[which];
  const float Ef = (float)E;
  const int64_t step = s->step;
  const int NE = B * B;
  for (int64_t q = (int64_t)blockIdx.x * POLY_WARPS + warp; q < nnzb; q += (int64_t)gridDim.x * POLY_WARPS) {
    const bool diag = rowidx[q] == col[q];
    for (int e = lane; e < NE; e += 32) {
      const int64_t idx = q * NE + e;
      double2 u;
      if (tail && deg >= 1) {
        float2 t = T.v[deg][idx];
        for (int m = deg - 1; m >= 1; --m) {
          const float2 vm = T.v[m][idx];
          t = make_float2(fmaf(t.x, Ef, vm.x), fmaf(t.y, Ef, vm.y));
        }
        const double2 v0 = V.v[0][idx];
        u = make_double2(fma((double)t.x, E, v0.x), fma((double)t.y, E, v0.y));
      } else {
        u = V.v[deg][idx];
        for (int m = deg - 1; m >= 0; --m) {
          const double2 vm = V.v[m][idx];
          u = make_double2(fma(u.x, E, vm.x), fma(u.y, E, vm.y));
        }
      }
      if (U) U[idx] = u;
      if (dU) store_du_block(tiles[warp], u, e, B, rs, q, diag, stochastic, step, idx, planar ? nullptr : dU);
    }
    __syncwarp();
    if (dU && planar) store_planar_block(tiles[warp], lane, q, dU);
    if (dU && dUH) store_dagger_block(tiles[warp], lane, B, rs, q, dUH);
    __syncwarp();
  }
}

void launch_field_poly(const PolyTerms& V, int deg, const DevState* s, int which, double2* U, float2* dU,
                       float2* dUH, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B, cudaStream_t st,
                       bool stochastic, bool planar, const PolyTerms32* tail) {
  RT_REQUIRE(deg >= 0 && deg < RT_MAX_POLY, RT_EINTERNAL, "field polynomial degree out of range");
  RT_REQUIRE(B <= 13, RT_EINTERNAL, "block size above 13");
  RT_REQUIRE(!planar || B == 13, RT_EINTERNAL, "column-planar blocks are 13-function blocks");
  RT_REQUIRE(!tail || (dU && !U && stochastic), RT_EINTERNAL,
             "the FP32 tail serves the stochastically rounded dU only");
  if (nnzb == 0) return;
  PolyTerms32 T;
  memset(&T, 0, sizeof(T));
  if (tail) T = *tail;
  k_field_poly<<<(unsigned)poly_grid(nnzb), POLY_WARPS * 32, 0, st>>>(V, deg, s, which, U, dU, dUH, nnzb, rowidx, col,
                                                                      B, rs32(B), stochastic ? 1 : 0, planar ? 1 : 0,
                                                                      T, tail ? 1 : 0);
  RT_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// FP32 Hotelling iterations of the CN propagator (mixed mode)
// ---------------------------------------------------------------------------
// Y <- 2I - Y on P_U, FP32 complex in the FP32 block layout (in place)
__global__ void k_two_i_minus32(float2* __restrict__ Y, int64_t nnzb, const int32_t* __restrict__ rowidx,
                                const int32_t* __restrict__ col, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx / NE;
    const int e = (int)(idx - q * NE);
    const int r = e / B, c = e - r * B;
    const int64_t o = q * (int64_t)B * rs + r * rs + c;
    const float d = (rowidx[q] == col[q] && r == c) ? 2.f : 0.f;
    const float2 y = Y[o];
    Y[o] = make_float2(d - y.x, -y.y);
  }
}

void launch_two_i_minus32(float2* Y, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B,
                          cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_two_i_minus32<<<(unsigned)g, 256, 0, st>>>(Y, nnzb, rowidx, col, B, rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

// FP32 complex blocks (FP32 block layout) to FP64 complex dense blocks
__global__ void k_f2d_unpad(const float2* __restrict__ a, double2* __restrict__ b, int64_t nnzb, int B, int rs) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NE = (int64_t)B * B;
  for (; idx < nnzb * NE; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx / NE;
    const int e = (int)(idx - q * NE);
    const int r = e / B, c = e - r * B;
    const float2 v = a[q * (int64_t)B * rs + r * rs + c];
    b[idx] = make_double2((double)v.x, (double)v.y);
  }
}

void launch_f2d_unpad(const float2* a, double2* b, int64_t nnzb, int B, cudaStream_t st) {
  int64_t n = nnzb * B * B;
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_f2d_unpad<<<(unsigned)g, 256, 0, st>>>(a, b, nnzb, B, rs32(B));
  RT_CUDA_CHECK(cudaGetLastError());
}

}  // namespace rt
