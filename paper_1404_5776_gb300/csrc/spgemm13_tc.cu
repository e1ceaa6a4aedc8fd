// Complex block products of 13-function atoms on the fifth-generation tensor
// cores (tcgen05), FP32-accurate through a 3xTF32 split.
//
// Same contraction as the FP32 CUDA-core kernels, C_ij = sum_k A_ik B_kj over
// the triple list of every output block, organised for the tensor cores:
//  * a tile is up to 8 consecutive output blocks (i, j_1..j_8) of one block
//    row; for every k the tile's items use (its "entries", the merged list),
//    one block MMA adds the contribution of A_ik to all of them at once:
//        D[(n, c)][(p, r)] += sum_kappa X[(n, c)][kappa] Y[kappa][(p, r)]
//    with M = 128 rows (n = item slot, c = column of the output block), N = 32
//    (p = real/imaginary part, r = row of the output block) and K = 32 (the
//    real and imaginary parts of the inner index m):
//        X = [Re B^T | Im B^T] of the items' B_kj, stacked,
//        Y = [[Re A^T, Im A^T], [-Im A^T, Re A^T]] of the shared A_ik,
//    the real form of a complex product, so D holds the real and imaginary
//    parts of C^T for the 8 blocks (13 x 13 blocks padded to 16 x 16);
//  * X lives in tensor memory (every thread writes its row with tcgen05.st),
//    Y in shared memory in the canonical K-major layout without swizzle
//    (core matrices of 8 rows x 16 B; K-direction stride 128 B, row-group
//    stride 1024 B), D in tensor memory;
//  * FP32 accuracy: every operand is split into a TF32 part and the FP32
//    remainder, and three MMAs per K step accumulate hi*hi + lo*hi + hi*lo.
//    The tensor cores' accumulation over many K steps is coarser than FP32
//    (measured: 2e-6 rms relative error over K = 1024 against 1.5e-7 for
//    sequential FP32 FMA), so it is kept to one entry (K = 32, where it
//    matches FP32): each entry writes a fresh accumulator (two alternate) and
//    the threads add the previous one into FP32 registers while the MMAs of
//    the next run;
//  * one elected thread issues the MMAs and commits them to an mbarrier; every
//    wait on it is bounded in time (the launch's budget), after which the
//    kernel records an error code, waits (bounded) for its MMAs in flight,
//    frees its tensor memory and returns;
//  * 128 threads per CTA over a persistent grid of tiles, 128 tensor-memory
//    columns per CTA; the dynamic shared memory request caps an SM at 4 CTAs,
//    so its 512 columns always suffice and no allocation waits.
#include "rt_internal.cuh"
#include "rt_ptx.cuh"

namespace rt {

namespace tc {

constexpr int BS = 13;
constexpr int RS = 16;
constexpr int SB = BS * RS;  // FP32 padded block (elements)
constexpr int NE = BS * BS;
constexpr int THREADS = 128;
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t COL_D0 = 0, COL_D1 = 32, COL_XH = 64, COL_XL = 96;
constexpr int SMEM_BYTES = 48 * 1024;
constexpr int OFF_YH = 0, OFF_YL = 4096, OFF_CTL = 8192, OFF_DIAG = 9216;
static_assert(OFF_DIAG + NE * 16 <= SMEM_BYTES, "shared memory layout");
static_assert(4 * TMEM_COLS <= 512 && (227 * 1024) / (SMEM_BYTES + 1024) <= 4, "tensor memory per SM");
constexpr long long DRAIN_NS = 2000000000ll;
// kind::tf32 instruction descriptor: D in F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// float index of element (row, k) of a 32 x 32 K-major tile in the canonical layout
__device__ __forceinline__ int canon(int row, int k) {
  return (((row >> 3) * 8 + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}
// shared-memory matrix descriptor: start address, K-direction core stride
// (128 B) and row-group stride (1024 B), all in 16-byte units; version 1;
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// D[tmem d] (+)= A[tmem a] * B[smem desc b]
__device__ __forceinline__ void mma(uint32_t d, uint32_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d),
      "r"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 columns of this thread's lane
__device__ __forceinline__ void st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}
__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
        "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
        "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Y element (row, kappa) of the canonical tiles: TF32 part and remainder
__device__ __forceinline__ void put_y(float* sYh, float* sYl, int row, int kap, float v) {
  const float h = tf32_hi(v);
  const int o = canon(row, kap);
  sYh[o] = h;
  sYl[o] = v - h;
}

template <int EPI>
__global__ void __launch_bounds__(THREADS) k_gemm13_c32_tc(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float* sYh = reinterpret_cast<float*>(sm + OFF_YH);
  float* sYl = reinterpret_cast<float*>(sm + OFF_YL);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + OFF_CTL);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_CTL + 8);
  double2* sdiag = reinterpret_cast<double2*>(sm + OFF_DIAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < (OFF_CTL / 4); i += THREADS) reinterpret_cast<float*>(sm)[i] = 0.f;  // padding stays zero
  if (tid == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tslot);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const float2* __restrict__ A = static_cast<const float2*>(g.A);
  const float2* __restrict__ Bm = static_cast<const float2*>(g.B);
  const int slot = tid >> 4, c = tid & 15;  // this thread's row of X and of D: item slot, output column
  // the Y elements (r, m) this thread converts: tid and tid + 128 (< 169)
  const int yr0 = tid / BS, ym0 = tid - BS * yr0;
  const int yr1 = (tid + THREADS) / BS, ym1 = tid + THREADS - BS * yr1;
  const bool has_y1 = tid + THREADS < NE;
  unsigned phase = 0;
  bool pending = false;  // committed MMAs not yet waited for
  int status = 0;        // 1: a wait expired

  for (int64_t t = blockIdx.x; t < g.tl_n; t += gridDim.x) {
    const int64_t e0 = g.tl_uptr[t], e1 = g.tl_uptr[t + 1];
    const int nit = g.tl_nitem[t];
    const int it0 = g.tl_item0[t];
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    float2 xv[BS], y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
    auto load = [&](int64_t e) {
      const int64_t ab = (int64_t)g.tl_ua[e] * SB;
      y0 = A[ab + yr0 * RS + ym0];
      if (has_y1) y1 = A[ab + yr1 * RS + ym1];
      const int bb = slot < nit ? g.tl_ub[e * TC_TILE + slot] : -1;
      if (bb >= 0 && c < BS) {
#pragma unroll
        for (int m = 0; m < BS; ++m) xv[m] = Bm[(int64_t)bb * SB + m * RS + c];
      } else {
#pragma unroll
        for (int m = 0; m < BS; ++m) xv[m] = make_float2(0.f, 0.f);
      }
    };
    if (e0 < e1) load(e0);
    for (int64_t e = e0; e < e1; ++e) {
      const int buf = (int)((e - e0) & 1);
      // the MMAs of the previous entry read X and Y: wait for them (bounded, CTA-wide verdict)
      const bool ok = pending ? mbar_wait(mbar, phase, g.wait_ns) : true;
      if (__syncthreads_or(!ok)) {
        status = 1;
        break;
      }
      if (pending) {
        phase ^= 1u;
        pending = false;
      }
      fence_after();
      // X row (slot, c) into tensor memory: TF32 parts and remainders
      {
        float xh[32], xl[32];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const float re = m < BS ? xv[m < BS ? m : 0].x : 0.f;
          const float im = m < BS ? xv[m < BS ? m : 0].y : 0.f;
          const float hr = tf32_hi(re), hi = tf32_hi(im);
          xh[m] = hr;
          xl[m] = re - hr;
          xh[16 + m] = hi;
          xl[16 + m] = im - hi;
        }
        st32(tmem + lane_base + COL_XH, xh);
        st32(tmem + lane_base + COL_XL, xl);
      }
      // Y = [[Re A^T, Im A^T], [-Im A^T, Re A^T]] as rows (p, r), columns (q, m)
      put_y(sYh, sYl, yr0, ym0, y0.x);
      put_y(sYh, sYl, yr0, 16 + ym0, -y0.y);
      put_y(sYh, sYl, 16 + yr0, ym0, y0.y);
      put_y(sYh, sYl, 16 + yr0, 16 + ym0, y0.x);
      if (has_y1) {
        put_y(sYh, sYl, yr1, ym1, y1.x);
        put_y(sYh, sYl, yr1, 16 + ym1, -y1.y);
        put_y(sYh, sYl, 16 + yr1, ym1, y1.y);
        put_y(sYh, sYl, 16 + yr1, 16 + ym1, y1.x);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      fence_proxy_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        const uint32_t d = tmem + (buf ? COL_D1 : COL_D0);
        const uint32_t yh = smem_u32(sYh), yl = smem_u32(sYl);
#pragma unroll
        for (int p = 0; p < 3; ++p) {  // hi*hi, lo*hi, hi*lo
          const uint32_t xa = tmem + (p == 1 ? COL_XL : COL_XH);
          const uint32_t yb = p == 2 ? yl : yh;
#pragma unroll
          for (int s = 0; s < 4; ++s) mma(d, xa + 8u * s, smem_desc(yb + 256u * s), (p | s) ? 1u : 0u);
        }
        commit(mbar);
      }
      pending = true;
      // the previous entry's accumulator (its MMAs are complete) into FP32 registers
      if (e > e0) {
        float v[32];
        ld32(tmem + lane_base + (buf ? COL_D0 : COL_D1), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += v[j];
      }
      fence_before();
      if (e + 1 < e1) load(e + 1);
    }
    if (status) break;
    if (e0 < e1) {
      const bool ok = pending ? mbar_wait(mbar, phase, g.wait_ns) : true;
      if (__syncthreads_or(!ok)) {
        status = 1;
        break;
      }
      if (pending) {
        phase ^= 1u;
        pending = false;
      }
      fence_after();
      float v[32];
      ld32(tmem + lane_base + (((e1 - 1 - e0) & 1) ? COL_D1 : COL_D0), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] += v[j];
      fence_before();
    }

    // epilogue: this thread holds column c of output block `slot`: acc[r] + i acc[16 + r]
    const bool valid = slot < nit && c < BS;
    const int q = valid ? g.item_blk[it0 + slot] : 0;
    if constexpr (EPI == EPI_STORE) {
      if (valid) {
        float2* __restrict__ C = static_cast<float2*>(g.C);
#pragma unroll
        for (int r = 0; r < BS; ++r) C[(int64_t)q * SB + r * RS + c] = make_float2(acc[r], acc[16 + r]);
        if (g.base) {  // delta form: W = K + M (K in FP64, dense blocks, through the map to K's pattern)
          const double2* __restrict__ Kb = static_cast<const double2*>(g.base);
          float2* __restrict__ W = static_cast<float2*>(g.U);
          const int kq = g.add_map ? g.add_map[q] : q;
#pragma unroll
          for (int r = 0; r < BS; ++r) {
            const double2 kv = kq >= 0 ? Kb[(int64_t)kq * NE + r * BS + c] : make_double2(0.0, 0.0);
            W[(int64_t)q * SB + r * RS + c] =
                make_float2((float)((double)acc[r] + kv.x), (float)((double)acc[16 + r] + kv.y));
          }
        }
      }
    } else {
      // K'_ij = K_ij (+ R_ij) + M_ij + acc for the upper blocks, mirrored;
      // the diagonal block made hermitian through shared memory
      int dslot = -1;
      for (int n = 0; n < nit; ++n) {
        const int qn = g.item_blk[it0 + n];
        if (g.rowidx[qn] == g.colidx[qn]) dslot = n;
      }
      double2* __restrict__ K = static_cast<double2*>(g.C);
      if (valid) {
        const double2* __restrict__ base = static_cast<const double2*>(g.base);
        const double2* __restrict__ R = static_cast<const double2*>(g.base2);
        const float2* __restrict__ add = static_cast<const float2*>(g.addend);
        const int aq = g.add_map ? g.add_map[q] : q;
        const bool diag = slot == dslot;
        const int qt = g.tmap[q];
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          double2 val = base[(int64_t)q * NE + r * BS + c];
          if (R) {
            const double2 rv = R[(int64_t)q * NE + r * BS + c];
            val = make_double2(val.x + rv.x, val.y + rv.y);
          }
          const float2 mv = aq >= 0 ? add[(int64_t)aq * SB + r * RS + c] : make_float2(0.f, 0.f);
          val = make_double2(val.x + ((double)mv.x + (double)acc[r]), val.y + ((double)mv.y + (double)acc[16 + r]));
          if (diag) {
            sdiag[r * BS + c] = val;
          } else {
            K[(int64_t)q * NE + r * BS + c] = val;
            K[(int64_t)qt * NE + c * BS + r] = make_double2(val.x, -val.y);
          }
        }
      }
      if (dslot >= 0) {
        __syncthreads();
        double herm = 0.0;
        if (valid && slot == dslot) {
#pragma unroll
          for (int r = 0; r < BS; ++r) {
            const double2 a = sdiag[r * BS + c], b = sdiag[c * BS + r];
            const double dr = a.x - b.x, di = a.y + b.y;
            herm = fmax(herm, sqrt(dr * dr + di * di));
            K[(int64_t)q * NE + r * BS + c] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
          }
        }
        for (int off = 16; off > 0; off >>= 1) herm = fmax(herm, __shfl_xor_sync(0xffffffffu, herm, off));
        if (lane == 0 && herm > 0.0 && g.herm_max)
          atomicMax(g.herm_max, (unsigned long long)__double_as_longlong(herm));
      }
    }
    __syncthreads();  // D read and the diagonal tile used by every thread before the next tile
  }

  if (status) {  // a wait expired: wait (bounded) for the MMAs in flight, then report
    int code = 1;
    if (pending && !mbar_wait(mbar, phase, DRAIN_NS)) code = 2;
    if (tid == 0 && g.err) atomicMax(g.err, code);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem);
}

// ---------------------------------------------------------------------------
// row tiles: merged A-block lists of up to TC_TILE items of one row
// ---------------------------------------------------------------------------
__global__ void k_tile_merge(const int64_t* __restrict__ ptr, const int2* __restrict__ ab,
                             const int32_t* __restrict__ item0, const int32_t* __restrict__ nitem, int64_t n_tiles,
                             int64_t* __restrict__ cnt, const int64_t* __restrict__ uptr, int32_t* __restrict__ ua,
                             int32_t* __restrict__ ub) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const int i0 = item0[t], n = nitem[t];
  int64_t p[TC_TILE], e[TC_TILE];
#pragma unroll
  for (int s = 0; s < TC_TILE; ++s) {
    p[s] = s < n ? ptr[i0 + s] : 0;
    e[s] = s < n ? ptr[i0 + s + 1] : 0;
  }
  int64_t out = uptr ? uptr[t] : 0, count = 0;
  for (;;) {
    int amin = 0x7fffffff;
#pragma unroll
    for (int s = 0; s < TC_TILE; ++s)
      if (p[s] < e[s]) amin = min(amin, ab[p[s]].x);
    if (amin == 0x7fffffff) break;
    if (ua) {
      ua[out] = amin;
#pragma unroll
      for (int s = 0; s < TC_TILE; ++s) {
        const bool hit = p[s] < e[s] && ab[p[s]].x == amin;
        ub[out * TC_TILE + s] = hit ? ab[p[s]].y : -1;
      }
      ++out;
    }
#pragma unroll
    for (int s = 0; s < TC_TILE; ++s)
      if (p[s] < e[s] && ab[p[s]].x == amin) ++p[s];
    ++count;
  }
  if (cnt) cnt[t] = count;
}

}  // namespace tc

void build_tiles(TileList& tl, const Triples& T, const Pattern& C, Arena& arena, cudaStream_t st) {
  using namespace tc;
  tl = TileList();
  const int64_t n_items = T.n_items;
  std::vector<int32_t> items(n_items);
  if (n_items)
    RT_CUDA_CHECK(cudaMemcpyAsync(items.data(), T.item_blk, sizeof(int32_t) * n_items, cudaMemcpyDeviceToHost, st));
  RT_CUDA_CHECK(cudaStreamSynchronize(st));
  std::vector<int32_t> h0, hn;
  int row = 0, cur = -1;
  for (int64_t it = 0; it < n_items; ++it) {
    const int q = items[it];
    while (row + 1 < (int)C.h_rowptr.size() && C.h_rowptr[row + 1] <= q) ++row;
    if (row != cur || hn.back() == TC_TILE) {
      h0.push_back((int32_t)it);
      hn.push_back(0);
      cur = row;
    }
    ++hn.back();
  }
  tl.n_tiles = (int64_t)h0.size();
  tl.item0 = arena.get_n<int32_t>(tl.n_tiles);
  tl.nitem = arena.get_n<int32_t>(tl.n_tiles);
  tl.uptr = arena.get_n<int64_t>(tl.n_tiles + 1);
  if (tl.n_tiles) {
    RT_CUDA_CHECK(cudaMemcpyAsync(tl.item0, h0.data(), sizeof(int32_t) * tl.n_tiles, cudaMemcpyHostToDevice, st));
    RT_CUDA_CHECK(cudaMemcpyAsync(tl.nitem, hn.data(), sizeof(int32_t) * tl.n_tiles, cudaMemcpyHostToDevice, st));
    Arena tmp;
    tmp.alloc = arena.alloc;
    tmp.stream = st;
    try {
      int64_t* cnt = tmp.get_n<int64_t>(tl.n_tiles + 1);
      const unsigned grid = (unsigned)((tl.n_tiles + 127) / 128);
      k_tile_merge<<<grid, 128, 0, st>>>(T.ptr, T.ab, tl.item0, tl.nitem, tl.n_tiles, cnt, nullptr, nullptr, nullptr);
      RT_CUDA_CHECK(cudaGetLastError());
      tl.n_entries = exclusive_scan_i64(cnt, tl.uptr, tl.n_tiles, tmp, st);
      tl.ua = arena.get_n<int32_t>(tl.n_entries);
      tl.ub = arena.get_n<int32_t>((size_t)tl.n_entries * TC_TILE);
      k_tile_merge<<<grid, 128, 0, st>>>(T.ptr, T.ab, tl.item0, tl.nitem, tl.n_tiles, nullptr, tl.uptr, tl.ua,
                                         tl.ub);
      RT_CUDA_CHECK(cudaGetLastError());
      RT_CUDA_CHECK(cudaStreamSynchronize(st));
    } catch (...) {
      cudaStreamSynchronize(st);
      tmp.release_all();
      throw;
    }
    tmp.release_all();
  } else {
    RT_CUDA_CHECK(cudaMemsetAsync(tl.uptr, 0, sizeof(int64_t), st));
  }
  tl.built = true;
}

bool launch_gemm13_tc(Epilogue epi, const GemmArgs& g, cudaStream_t st) {
  using namespace tc;
  if (epi != EPI_STORE && epi != EPI_DELTA_SANDWICH) return false;
  if (g.tl_n == 0) return true;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    RT_CUDA_CHECK(cudaGetDevice(&dev));
    RT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t grid = std::min<int64_t>(g.tl_n, (int64_t)sms * 4);
  if (epi == EPI_STORE)
    k_gemm13_c32_tc<EPI_STORE><<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(g);
  else
    k_gemm13_c32_tc<EPI_DELTA_SANDWICH><<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(g);
  RT_CUDA_CHECK(cudaGetLastError());
  return true;
}

}  // namespace rt
