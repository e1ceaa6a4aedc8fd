// FP32 block products for 4-function atoms (the mixed-precision path).
//
// Same contraction as spgemm.cu (C_ij = sum_k op(A)_ik op(B)_kj over the
// triple list of the output block, k ascending), laid out for 4 x 4 blocks:
//   * one lane owns one output block and keeps its 16 elements in registers;
//   * per triple the lane reads the whole A and B blocks with 16-byte loads
//     (64 B real / 128 B complex each, one cache line) and does 4^3 multiply-
//     adds; B^dagger is read transposed and conjugated from registers;
//   * global-load latency is hidden by occupancy (8 warps per block, every
//     lane independent), not by staging: a 4 x 4 block is too small for a
//     shared-memory pipeline to pay;
//   * epilogues are fused per lane: Taylor accumulation into U, store, add,
//     and the delta-form sandwich K' = K + M + W dU^dagger with the mirror
//     and the hermitian diagonal block.
#include <algorithm>

#include "rt_internal.cuh"

namespace rt {

namespace f32b4 {

constexpr int NE = 16;
constexpr int THREADS = 256;

__device__ __forceinline__ void load_block(const float* __restrict__ p, float (&v)[NE]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 f = q[k];
    v[4 * k] = f.x;
    v[4 * k + 1] = f.y;
    v[4 * k + 2] = f.z;
    v[4 * k + 3] = f.w;
  }
}
__device__ __forceinline__ void load_block(const float2* __restrict__ p, float2 (&v)[NE]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 f = q[k];
    v[2 * k] = make_float2(f.x, f.y);
    v[2 * k + 1] = make_float2(f.z, f.w);
  }
}
__device__ __forceinline__ void store_block(float* p, const float (&v)[NE]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
__device__ __forceinline__ void store_block(float2* p, const float2 (&v)[NE]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < 8; ++k) q[k] = make_float4(v[2 * k].x, v[2 * k].y, v[2 * k + 1].x, v[2 * k + 1].y);
}

__device__ __forceinline__ float fma_v(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 fma_v(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float conj_v(float a) { return a; }
__device__ __forceinline__ float2 conj_v(float2 a) { return make_float2(a.x, -a.y); }
template <typename V>
__device__ __forceinline__ V zero_v();
template <>
__device__ __forceinline__ float zero_v<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.f, 0.f); }

template <typename V, bool BDAG, int EPI>
__device__ __forceinline__ void g4_item(const GemmArgs& g, int64_t item) {
  const V* __restrict__ A = static_cast<const V*>(g.A);
  const V* __restrict__ B = static_cast<const V*>(g.B);
  V acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e] = zero_v<V>();
  const int64_t t0 = g.ptr[item], t1 = g.ptr[item + 1];
  for (int64_t t = t0; t < t1; ++t) {
    const int2 ab = g.ab[t];
    V a[NE], b[NE];
    load_block(A + (int64_t)ab.x * NE, a);
    load_block(B + (int64_t)ab.y * NE, b);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        V v = acc[r * 4 + c];
#pragma unroll
        for (int m = 0; m < 4; ++m) v = fma_v(a[r * 4 + m], BDAG ? conj_v(b[c * 4 + m]) : b[m * 4 + c], v);
        acc[r * 4 + c] = v;
      }
  }
  const int q = g.item_blk[item];
  if constexpr (EPI == EPI_STORE) {
    store_block(static_cast<V*>(g.C) + (int64_t)q * NE, acc);
    if constexpr (sizeof(V) == 8) {
      // delta form: also W = dK + M in FP32 (dK in FP64 through the map from
      // this pattern to dK's; -1 = no dK block), one rounding per element
      if (g.base) {
        const int kq = g.add_map ? g.add_map[q] : q;
        float2 w[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
          double2 kv = make_double2(0.0, 0.0);
          if (kq >= 0) kv = static_cast<const double2*>(g.base)[(int64_t)kq * NE + e];
          w[e] = make_float2((float)((double)acc[e].x + kv.x), (float)((double)acc[e].y + kv.y));
        }
        store_block(static_cast<float2*>(g.U) + (int64_t)q * NE, w);
      }
    }
  } else if constexpr (EPI == EPI_ADD) {
    V* C = static_cast<V*>(g.C) + (int64_t)q * NE;
    V old[NE];
    load_block(C, old);
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if constexpr (sizeof(V) == 4) acc[e] = old[e] + acc[e];
      else acc[e] = make_float2(old[e].x + acc[e].x, old[e].y + acc[e].y);
    }
    store_block(C, acc);
  } else if constexpr (EPI == EPI_STORE_ACC) {
    // real power T^n stored (unless C is null); coef * T^n added to complex U
    if constexpr (sizeof(V) == 4) {
      if (g.C) store_block(static_cast<float*>(g.C) + (int64_t)q * NE, acc);
      const int uq = g.umap ? g.umap[q] : q;
      if (uq >= 0) {
        float2* U = static_cast<float2*>(g.U) + (int64_t)uq * NE;
        float2 u[NE];
        load_block(U, u);
        const float cf = (float)g.coef;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
          if (g.coef_imag) u[e].y += cf * acc[e];
          else u[e].x += cf * acc[e];
        }
        store_block(U, u);
      }
    }
  } else if constexpr (EPI == EPI_DELTA_SANDWICH) {
    if constexpr (sizeof(V) == 8) {
      // K'_ij = K_ij (+ R_ij) + M_ij + acc for j >= i (K in FP64); mirror; hermitian diagonal
      const int i = g.rowidx[q], j = g.colidx[q];
      double2* __restrict__ K = static_cast<double2*>(g.C);
      const double2* __restrict__ base = static_cast<const double2*>(g.base) + (int64_t)q * NE;
      const int aq = g.add_map ? g.add_map[q] : q;
      float2 mv[NE];
      if (aq >= 0) load_block(static_cast<const float2*>(g.addend) + (int64_t)aq * NE, mv);
      else
#pragma unroll
        for (int e = 0; e < NE; ++e) mv[e] = make_float2(0.f, 0.f);
      const int qt = g.tmap[q];
      // reference split: R = U K_ref U^dagger - K_ref (FP64) joins the base
      const double2* __restrict__ R = g.base2 ? static_cast<const double2*>(g.base2) + (int64_t)q * NE : nullptr;
      // or R(E) = sum_p E^p B_p at this step's field, by Horner here
      const double E = g.rpoly ? *g.poly_E : 0.0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int e = r * 4 + c;
          double2 kv = base[e];
          if (R) {
            kv = make_double2(kv.x + R[e].x, kv.y + R[e].y);
          } else if (g.rpoly) {
            const int64_t idx = (int64_t)q * NE + e;
            double2 rv = g.rpoly[g.rdeg][idx];
            for (int p = g.rdeg - 1; p >= 0; --p) {
              const double2 cp = g.rpoly[p][idx];
              rv = make_double2(fma(rv.x, E, cp.x), fma(rv.y, E, cp.y));
            }
            kv = make_double2(kv.x + rv.x, kv.y + rv.y);
          }
          const double2 v =
              make_double2(kv.x + ((double)mv[e].x + (double)acc[e].x), kv.y + ((double)mv[e].y + (double)acc[e].y));
          K[(int64_t)q * NE + e] = v;
          if (i != j) K[(int64_t)qt * NE + c * 4 + r] = make_double2(v.x, -v.y);
          if (g.kf32 && i != j) {
            float2* __restrict__ Kf = static_cast<float2*>(g.kf32);
            Kf[(int64_t)q * NE + e] = make_float2((float)v.x, (float)v.y);
            Kf[(int64_t)qt * NE + c * 4 + r] = make_float2((float)v.x, (float)-v.y);
          }
        }
      if (i == j) {
        // diagonal block (one item in ~100): read the lane's own stores back,
        // then write (K' + K'^dagger)/2 and record |K' - K'^dagger|
        double2 v[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) v[e] = K[(int64_t)q * NE + e];
        double herm = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const double2 a = v[r * 4 + c], t = v[c * 4 + r];
            const double dr = a.x - t.x, di = a.y + t.y;
            herm = fmax(herm, sqrt(dr * dr + di * di));
            const double2 w = make_double2(0.5 * (a.x + t.x), 0.5 * (a.y - t.y));
            K[(int64_t)q * NE + r * 4 + c] = w;
            if (g.kf32)
              static_cast<float2*>(g.kf32)[(int64_t)q * NE + r * 4 + c] = make_float2((float)w.x, (float)w.y);
          }
        if (g.herm_max) atomicMax(g.herm_max, (unsigned long long)__double_as_longlong(herm));
      }
    }
  }
}

// One lane per item (output block); a persistent launch (g.persistent) walks
// items with a grid-wide stride, and a grouped launch (g.grp) takes item i as
// item gitems[i].y of the product described by grp[gitems[i].x].
template <typename V, bool BDAG, int EPI>
__global__ void __launch_bounds__(THREADS, 2) k_gemm4_f32(const __grid_constant__ GemmArgs g) {
  int64_t item = (int64_t)blockIdx.x * THREADS + threadIdx.x;
  const int64_t stride = g.persistent ? (int64_t)gridDim.x * THREADS : g.n_items;
  for (; item < g.n_items; item += stride) {
    const int2 gi = g.grp ? g.gitems[item] : make_int2(0, 0);
    g4_item<V, BDAG, EPI>(g.grp ? g.grp[gi.x] : g, g.grp ? (int64_t)gi.y : item);
  }
}

template <typename V, bool BDAG, int EPI>
void launch_one(const GemmArgs& g, cudaStream_t st) {
  int64_t grid = (g.n_items + THREADS - 1) / THREADS;
  if (g.persistent) {
    int dev = 0, sms = 0;
    RT_CUDA_CHECK(cudaGetDevice(&dev));
    RT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grid = std::min<int64_t>(grid, (int64_t)sms * 2);  // 2 CTAs per SM (launch bounds)
  }
  RT_REQUIRE(grid < (1ll << 31), RT_EINTERNAL, "grid too large");
  k_gemm4_f32<V, BDAG, EPI><<<(unsigned)grid, THREADS, 0, st>>>(g);
  RT_CUDA_CHECK(cudaGetLastError());
}

}  // namespace f32b4

// Launches the FP32 kernels for 4-function blocks; false if the variant is
// not one of theirs (the generic kernel then runs it).
bool launch_gemm4_f32(bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g, cudaStream_t st) {
  using namespace f32b4;
  RT_REQUIRE(!(g.grp || g.persistent) || cplx, RT_EINTERNAL, "grouped and persistent launches are complex products");
  RT_REQUIRE(!g.base || (cplx && !b_dag && epi == EPI_STORE) || epi == EPI_DELTA_SANDWICH, RT_EINTERNAL,
             "W = dK + M comes with the complex store epilogue");
  if (a_dag) return false;
  if (g.n_items == 0) return true;
  if (!cplx) {
    if (b_dag) return false;
    if (epi == EPI_STORE) return launch_one<float, false, EPI_STORE>(g, st), true;
    if (epi == EPI_STORE_ACC) return launch_one<float, false, EPI_STORE_ACC>(g, st), true;
    if (epi == EPI_ADD) return launch_one<float, false, EPI_ADD>(g, st), true;
    return false;
  }
  if (!b_dag) {
    if (epi == EPI_STORE) return launch_one<float2, false, EPI_STORE>(g, st), true;
    if (epi == EPI_ADD) return launch_one<float2, false, EPI_ADD>(g, st), true;
    return false;
  }
  if (epi == EPI_STORE) return launch_one<float2, true, EPI_STORE>(g, st), true;
  if (epi == EPI_DELTA_SANDWICH) return launch_one<float2, true, EPI_DELTA_SANDWICH>(g, st), true;
  return false;
}

}  // namespace rt
