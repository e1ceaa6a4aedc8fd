// Truncated block-sparse products C = cut_{P_C}(op(A) op(B)).
//
// Every product of the step (paper Sec. II.A cut-off; T = S^-1 H, the Taylor
// powers of eq. matrix_exp, the sandwich of the formal solution
// K(t) = U K U^dagger, Hotelling's iteration of Sec. V.A) is a sum over block
// triples: C_ij = sum_k op(A)_ik op(B)_kj for (i,j) in P_C, k ascending.  The
// triple lists are built once (atoms are stationary).
//
// Thread mapping: a group of LPB lanes owns one output block; each lane owns
// EPL of its B*B elements and keeps them in registers.  Per triple the group
// stages op(A)_ik and op(B)_kj (conjugate transposes applied on the way into
// shared memory) and every lane accumulates its elements over the block's inner
// index.  Epilogues are fused: Taylor accumulation into U, the Hotelling
// 2I - AX step with its residual, and the hermitian mirror of K' = M U^dagger.
#include "rt_internal.cuh"

namespace rt {

template <typename E>
struct CT;
template <>
struct CT<double> {
  using R = double;
  using C = double2;
};
template <>
struct CT<float> {
  using R = float;
  using C = float2;
};

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double cfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float cfma(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double2 conjv(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 conjv(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double conjv(double a) { return a; }
__device__ __forceinline__ float conjv(float a) { return a; }

template <typename T>
__device__ __forceinline__ T zero_v();
template <>
__device__ __forceinline__ double zero_v<double>() { return 0.0; }
template <>
__device__ __forceinline__ float zero_v<float>() { return 0.f; }
template <>
__device__ __forceinline__ double2 zero_v<double2>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double re_of(double a) { return a; }
__device__ __forceinline__ double re_of(float a) { return a; }
__device__ __forceinline__ double re_of(double2 a) { return a.x; }
__device__ __forceinline__ double re_of(float2 a) { return a.x; }
__device__ __forceinline__ double im_of(double) { return 0.0; }
__device__ __forceinline__ double im_of(float) { return 0.0; }
__device__ __forceinline__ double im_of(double2 a) { return a.y; }
__device__ __forceinline__ double im_of(float2 a) { return a.y; }

template <typename T>
__device__ __forceinline__ T make_v(double re, double im);
template <>
__device__ __forceinline__ double make_v<double>(double re, double) { return re; }
template <>
__device__ __forceinline__ float make_v<float>(double re, double) { return (float)re; }
template <>
__device__ __forceinline__ double2 make_v<double2>(double re, double im) { return make_double2(re, im); }
template <>
__device__ __forceinline__ float2 make_v<float2>(double re, double im) { return make_float2((float)re, (float)im); }

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

template <int BS>
struct Map {
  static constexpr int NE = BS * BS;
  static constexpr int LPB = (BS == 1) ? 1 : (NE <= 16 ? 16 : 32);
  static constexpr int EPL = (NE + LPB - 1) / LPB;
  static constexpr int GPW = 32 / LPB;  // groups per warp
};

template <int LPB>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (LPB == 32) return 0xffffffffu;
  else if constexpr (LPB == 16) return (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  else return 1u << (threadIdx.x & 31);
}

template <int LPB>
__device__ __forceinline__ void group_sync() {
  if constexpr (LPB == 32) {
    __syncwarp();
  } else if constexpr (LPB == 16) {
    unsigned mask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
    __syncwarp(mask);
  }
}

constexpr int GEMM_WARPS = 8;

template <int BS, typename V, bool ADAG, bool BDAG, int EPI>
__global__ void __launch_bounds__(GEMM_WARPS * 32) k_gemm(GemmArgs g) {
  using M = Map<BS>;
  constexpr int NE = M::NE, LPB = M::LPB, EPL = M::EPL;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int grp_in_warp = lane / LPB;
  const int gl = lane % LPB;  // lane within group
  const int64_t groups_per_cta = GEMM_WARPS * M::GPW;
  const int64_t item = (int64_t)blockIdx.x * groups_per_cta + warp * M::GPW + grp_in_warp;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sA = reinterpret_cast<V*>(smem_raw) + (warp * M::GPW + grp_in_warp) * (2 * NE);
  V* sB = sA + NE;

  const bool active = item < g.n_items;
  V acc[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) acc[e] = zero_v<V>();

  const V* __restrict__ A = static_cast<const V*>(g.A);
  const V* __restrict__ B = static_cast<const V*>(g.B);

  int64_t t0 = 0, t1 = 0;
  if (active) {
    t0 = g.ptr[item];
    t1 = g.ptr[item + 1];
  }
  for (int64_t t = t0; t < t1; ++t) {
    int2 ab = g.ab[t];
    const V* a = A + (int64_t)ab.x * NE;
    const V* b = B + (int64_t)ab.y * NE;
    if constexpr (BS == 1) {
      V av = ADAG ? conjv(a[0]) : a[0];
      V bv = BDAG ? conjv(b[0]) : b[0];
      acc[0] = cfma(av, bv, acc[0]);
    } else {
      for (int e = gl; e < NE; e += LPB) {
        int x = e / BS, y = e - x * BS;
        V av = a[e];
        V bv = b[e];
        if (ADAG) sA[y * BS + x] = conjv(av);
        else sA[e] = av;
        if (BDAG) sB[y * BS + x] = conjv(bv);
        else sB[e] = bv;
      }
      group_sync<LPB>();
#pragma unroll
      for (int s = 0; s < EPL; ++s) {
        int e = gl + s * LPB;
        if (e < NE) {
          int r = e / BS, c = e - r * BS;
          V v = acc[s];
#pragma unroll
          for (int m = 0; m < BS; ++m) v = cfma(sA[r * BS + m], sB[m * BS + c], v);
          acc[s] = v;
        }
      }
      group_sync<LPB>();
    }
  }
  if (!active) return;

  const int q = g.item_blk[item];
  V* __restrict__ C = static_cast<V*>(g.C);

  if constexpr (EPI == EPI_STORE) {
#pragma unroll
    for (int s = 0; s < EPL; ++s) {
      int e = gl + s * LPB;
      if (e < NE) C[(int64_t)q * NE + e] = acc[s];
    }
  } else if constexpr (EPI == EPI_ADD) {
#pragma unroll
    for (int s = 0; s < EPL; ++s) {
      int e = gl + s * LPB;
      if (e < NE) {
        V old = C[(int64_t)q * NE + e];
        C[(int64_t)q * NE + e] = make_v<V>(re_of(old) + re_of(acc[s]), im_of(old) + im_of(acc[s]));
      }
    }
  } else if constexpr (EPI == EPI_STORE_ACC) {
    // real power T^n (V real) stored; coef * T^n added to complex U
    using CV = typename CT<V>::C;
    CV* __restrict__ U = static_cast<CV*>(g.U);
    int uq = g.umap ? g.umap[q] : q;
#pragma unroll
    for (int s = 0; s < EPL; ++s) {
      int e = gl + s * LPB;
      if (e < NE) {
        if (C) C[(int64_t)q * NE + e] = acc[s];  // null: power needed only inside U
        if (uq >= 0) {
          CV u = U[(int64_t)uq * NE + e];
          if (g.coef_imag) u.y += (decltype(u.y))(g.coef * re_of(acc[s]));
          else u.x += (decltype(u.x))(g.coef * re_of(acc[s]));
          U[(int64_t)uq * NE + e] = u;
        }
      }
    }
  } else if constexpr (EPI == EPI_TWO_I) {
    const int i = g.rowidx[q], j = g.colidx[q];
    const int bi = g.bsize[i], bj = g.bsize[j];
    double part = 0.0;
#pragma unroll
    for (int s = 0; s < EPL; ++s) {
      int e = gl + s * LPB;
      if (e < NE) {
        int r = e / BS, c = e - r * BS;
        double dre = ((i == j && r == c) ? 1.0 : 0.0) - re_of(acc[s]);
        double dim = -im_of(acc[s]);
        if (r < bi && c < bj) part += dre * dre + dim * dim;
        double two = (i == j && r == c) ? 2.0 : 0.0;
        C[(int64_t)q * NE + e] = make_v<V>(two - re_of(acc[s]), -im_of(acc[s]));
      }
    }
    // group reduction of the residual part (fixed order)
#pragma unroll
    for (int off = LPB / 2; off > 0; off >>= 1) part += __shfl_down_sync(group_mask<LPB>(), part, off, LPB);
    if (gl == 0) g.red[item] = part;
  } else if constexpr (EPI == EPI_SANDWICH || EPI == EPI_DELTA_SANDWICH) {
    // K'_ij for j >= i; mirror K'_ji = K'_ij^dagger; hermitian diagonal blocks
    const int i = g.rowidx[q], j = g.colidx[q];
    using KV = typename CT<double>::C;  // K is always complex FP64
    KV* __restrict__ K = static_cast<KV*>(g.C);
    KV val[EPL];
#pragma unroll
    for (int s = 0; s < EPL; ++s) {
      int e = gl + s * LPB;
      val[s] = make_double2(0.0, 0.0);
      if (e < NE) {
        double vr = re_of(acc[s]), vi = im_of(acc[s]);
        if constexpr (EPI == EPI_DELTA_SANDWICH) {
          const KV* base = static_cast<const KV*>(g.base);
          const V* add = static_cast<const V*>(g.addend);
          KV b0 = base[(int64_t)q * NE + e];
          int aq = g.add_map ? g.add_map[q] : q;
          double ar = 0.0, ai = 0.0;
          if (aq >= 0) {
            ar = re_of(add[(int64_t)aq * NE + e]);
            ai = im_of(add[(int64_t)aq * NE + e]);
          }
          vr = b0.x + (ar + vr);
          vi = b0.y + (ai + vi);
        }
        val[s] = make_double2(vr, vi);
      }
    }
    if (i != j) {
      const int qt = g.tmap[q];
#pragma unroll
      for (int s = 0; s < EPL; ++s) {
        int e = gl + s * LPB;
        if (e < NE) {
          int r = e / BS, c = e - r * BS;
          K[(int64_t)q * NE + e] = val[s];
          K[(int64_t)qt * NE + c * BS + r] = make_double2(val[s].x, -val[s].y);
        }
      }
    } else {
      // stage the block in shared memory to pair (r,c) with (c,r)
      // reuse this group's own staging area (2*NE values >= NE complex doubles)
      double2* sK = reinterpret_cast<double2*>(sA);
      if constexpr (BS > 1) group_sync<LPB>();
#pragma unroll
      for (int s = 0; s < EPL; ++s) {
        int e = gl + s * LPB;
        if (e < NE) sK[e] = val[s];
      }
      if constexpr (BS > 1) group_sync<LPB>();
      double herm = 0.0;
#pragma unroll
      for (int s = 0; s < EPL; ++s) {
        int e = gl + s * LPB;
        if (e < NE) {
          int r = e / BS, c = e - r * BS;
          double2 tv = sK[c * BS + r];
          double dr = val[s].x - tv.x, di = val[s].y + tv.y;  // K - K^dagger
          herm = fmax(herm, sqrt(dr * dr + di * di));
          K[(int64_t)q * NE + e] = make_double2(0.5 * (val[s].x + tv.x), 0.5 * (val[s].y - tv.y));
        }
      }
      if (g.herm_max) atomic_max_nonneg(g.herm_max, herm);
    }
  }
}

template <int BS, typename V, bool ADAG, bool BDAG, int EPI>
static void launch_one(const GemmArgs& g, cudaStream_t st) {
  using M = Map<BS>;
  if (g.n_items == 0) return;
  int64_t groups_per_cta = GEMM_WARPS * M::GPW;
  int64_t grid = (g.n_items + groups_per_cta - 1) / groups_per_cta;
  size_t smem_v = (size_t)GEMM_WARPS * M::GPW * 2 * M::NE * sizeof(V);
  size_t smem = smem_v;
  if (EPI == EPI_SANDWICH || EPI == EPI_DELTA_SANDWICH)
    RT_REQUIRE(2 * sizeof(V) >= sizeof(double2), RT_EINTERNAL, "sandwich staging too small");
  if (smem < 16) smem = 16;
  if (smem > 48 * 1024) {
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm<BS, V, ADAG, BDAG, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
  }
  RT_REQUIRE(grid < (1ll << 31), RT_EINTERNAL, "grid too large");
  k_gemm<BS, V, ADAG, BDAG, EPI><<<(unsigned)grid, GEMM_WARPS * 32, smem, st>>>(g);
  RT_CUDA_CHECK(cudaGetLastError());
}

template <int BS, typename R>
static void dispatch_prec(bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g, cudaStream_t st) {
  using C = typename CT<R>::C;
  if (!cplx) {
    RT_REQUIRE(!a_dag && !b_dag, RT_EINTERNAL, "real products take no conjugate transpose");
    switch (epi) {
      case EPI_STORE: return launch_one<BS, R, false, false, EPI_STORE>(g, st);
      case EPI_STORE_ACC: return launch_one<BS, R, false, false, EPI_STORE_ACC>(g, st);
      case EPI_TWO_I: return launch_one<BS, R, false, false, EPI_TWO_I>(g, st);
      case EPI_ADD: return launch_one<BS, R, false, false, EPI_ADD>(g, st);
      default: break;
    }
  } else if (!a_dag && !b_dag) {
    switch (epi) {
      case EPI_STORE: return launch_one<BS, C, false, false, EPI_STORE>(g, st);
      case EPI_TWO_I: return launch_one<BS, C, false, false, EPI_TWO_I>(g, st);
      case EPI_ADD: return launch_one<BS, C, false, false, EPI_ADD>(g, st);
      default: break;
    }
  } else if (!a_dag && b_dag) {
    switch (epi) {
      case EPI_SANDWICH: return launch_one<BS, C, false, true, EPI_SANDWICH>(g, st);
      case EPI_DELTA_SANDWICH: return launch_one<BS, C, false, true, EPI_DELTA_SANDWICH>(g, st);
      case EPI_STORE: return launch_one<BS, C, false, true, EPI_STORE>(g, st);
      default: break;
    }
  } else if (a_dag && !b_dag) {
    if (epi == EPI_STORE) return launch_one<BS, C, true, false, EPI_STORE>(g, st);
  }
  throw Error{RT_EINTERNAL, "unsupported product variant"};
}

bool launch_gemm13_f32(bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g, cudaStream_t st);
bool launch_gemm4_f32(bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g, cudaStream_t st);

void launch_gemm(int B, bool fp32, bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g,
                 cudaStream_t st) {
  if (B == 13 && fp32) {
    // FP32 13-function matrices use the padded block layout of these kernels only
    if (launch_gemm13_f32(cplx, a_dag, b_dag, epi, g, st)) return;
    throw Error{RT_EINTERNAL, "FP32 13-function product variant has no kernel"};
  }
  if (B == 4 && fp32 && launch_gemm4_f32(cplx, a_dag, b_dag, epi, g, st)) return;
  switch (B) {
    case 1: return fp32 ? dispatch_prec<1, float>(cplx, a_dag, b_dag, epi, g, st)
                        : dispatch_prec<1, double>(cplx, a_dag, b_dag, epi, g, st);
    case 4: return fp32 ? dispatch_prec<4, float>(cplx, a_dag, b_dag, epi, g, st)
                        : dispatch_prec<4, double>(cplx, a_dag, b_dag, epi, g, st);
    case 13: return fp32 ? dispatch_prec<13, float>(cplx, a_dag, b_dag, epi, g, st)
                         : dispatch_prec<13, double>(cplx, a_dag, b_dag, epi, g, st);
    default: throw Error{RT_EINVAL, "block size must pad to 1, 4 or 13"};
  }
}

}  // namespace rt
