// FP32 block products for 13-function atoms (the mixed-precision path).
//
// Same contraction as spgemm.cu (C_ij = sum_k op(A)_ik op(B)_kj over the
// triple list of the output block, k ascending), laid out for FP32 throughput
// on the CUDA cores:
//   * FP32 matrices of 13-function atoms are stored with a padded row stride
//     of 16 (one block = 13 x 16 elements = 832 B real / 1664 B complex, 16 B
//     aligned), the same layout the blocks take in shared memory;
//   * one warp owns one 13x13 output block; one elected lane streams the A and
//     B blocks of the next NT triples into shared memory with 1D TMA bulk
//     copies (cp.async.bulk) completing on a per-stage mbarrier (two stages:
//     the next group is in flight while the current one is multiplied);
//   * the warp splits into NT lane groups that take interleaved triples
//     (complex: 2 groups of 16 lanes, real: 4 groups of 8 lanes); a lane keeps
//     one (complex) or two (real) output columns and the matching B column(s)
//     in registers and reads the A rows as shared-memory broadcasts;
//   * B^dagger operands are pre-transposed (a conjugate-transposed copy of
//     U - I), so every staged block is a straight copy;
//   * the groups' partial sums meet through warp shuffles at the end;
//   * every wait on an mbarrier is bounded: on expiry the kernel records an
//     error code, waits (bounded) for its copies in flight and returns.
#include "rt_internal.cuh"

namespace rt {

namespace f32 {

constexpr int BS = 13;
constexpr int NE = BS * BS;
constexpr int RS = 16;        // padded row stride
constexpr int SB = BS * RS;   // padded block (elements)
constexpr int WARPS = 4;
// One staged triple = A block + B block + 16 bytes of skew, so that the lane
// groups' broadcast reads of different triples fall on different banks.
template <typename V>
struct Slot {
  static constexpr int SKEW = 16 / sizeof(V);
  static constexpr int STRIDE = 2 * SB + SKEW;  // elements
};
constexpr long long SPIN_LIMIT = 1ll << 26;  // ~ seconds of polling before giving up

__device__ __forceinline__ float2 cfma2(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}

__device__ __forceinline__ void amax_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  unsigned addr = smem_u32(bar);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Issue the TMA copies of one group of NT triples into `buf` (slot k holds A
// at k*STRIDE and B at k*STRIDE + SB).  Lane 0 arms the stage's mbarrier with
// the byte count; then lanes 0..2NT-1 issue one bulk copy each (all copies in
// one warp-wide instruction).  `blk` is the lane's block index for this group,
// loaded one group ahead (-1: past the end, copy a zero block).
template <typename V, int NT>
__device__ __forceinline__ void issue_group(V* buf, const V* __restrict__ A, const V* __restrict__ B, int blk,
                                            const V* __restrict__ zero, uint64_t* bar, int lane) {
  constexpr unsigned BYTES = SB * sizeof(V);
  if (lane == 0) mbar_expect_tx(bar, NT * 2 * BYTES);
  __syncwarp();
  if (lane < 2 * NT) {
    const int k = lane >> 1;
    const bool isB = lane & 1;
    const V* src = blk < 0 ? zero : (isB ? B : A) + (int64_t)blk * SB;
    tma_load_1d(buf + k * Slot<V>::STRIDE + (isB ? SB : 0), src, BYTES, bar);
  }
}

// The block index lane `lane` (< 2NT) copies for the group starting at tb.
template <int NT>
__device__ __forceinline__ int group_block(const int2* __restrict__ ab, int64_t tb, int64_t t1, int lane) {
  if (lane >= 2 * NT) return -1;
  const int64_t t = tb + (lane >> 1);
  if (t >= t1) return -1;
  const int2 p = ab[t];
  return (lane & 1) ? p.y : p.x;
}

struct Smem {
  uint64_t bar[WARPS][2];
};

// ---------------------------------------------------------------------------
// complex: 2 groups x 16 lanes, lane (h, c) owns output column c (c < 13)
// ---------------------------------------------------------------------------
template <int EPI>
__global__ void __launch_bounds__(WARPS * 32, 4) k_gemm13_c32(GemmArgs g) {
  constexpr int NT = 2;
  constexpr int WBUF = NT * Slot<float2>::STRIDE;  // one stage of one warp (float2)
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int h = lane >> 4;
  const int c = lane & 15;
  const int64_t item = (int64_t)blockIdx.x * WARPS + warp;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  Smem* ctl = reinterpret_cast<Smem*>(dyn_smem);
  float2* wsm = reinterpret_cast<float2*>(dyn_smem + 128) + (size_t)warp * 2 * WBUF;
  if (item >= g.n_items) return;  // whole warp leaves together
  uint64_t* bar = ctl->bar[warp];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncwarp();

  const float2* __restrict__ A = static_cast<const float2*>(g.A);
  const float2* __restrict__ B = static_cast<const float2*>(g.B);
  const float2* __restrict__ Z = static_cast<const float2*>(g.zero);
  const int64_t t0 = g.ptr[item], t1 = g.ptr[item + 1];

  float2 acc[BS];
#pragma unroll
  for (int r = 0; r < BS; ++r) acc[r] = make_float2(0.f, 0.f);

  unsigned phase = 0u;    // bit s: parity to wait for on stage s
  unsigned pending = 0u;  // bit s: copies in flight into stage s
  bool ok = true;
  int stage = 0;
  int nblk = -1;  // this lane's block index for the next group (prefetched)
  if (t0 < t1) {
    issue_group<float2, NT>(wsm, A, B, group_block<NT>(g.ab, t0, t1, lane), Z, &bar[0], lane);
    nblk = group_block<NT>(g.ab, t0 + NT, t1, lane);
    pending |= 1u;
  }
  for (int64_t tb = t0; tb < t1; tb += NT) {
    if (tb + NT < t1) {
      issue_group<float2, NT>(wsm + (stage ^ 1) * WBUF, A, B, nblk, Z, &bar[stage ^ 1], lane);
      nblk = group_block<NT>(g.ab, tb + 2 * NT, t1, lane);  // used one iteration later
      pending |= 1u << (stage ^ 1);
    }
    if (!mbar_wait(&bar[stage], (phase >> stage) & 1u)) {
      ok = false;
      break;
    }
    phase ^= 1u << stage;
    pending &= ~(1u << stage);
    const float2* sA = wsm + stage * WBUF + h * Slot<float2>::STRIDE;
    const float2* sB = sA + SB;
    float2 bcol[BS];
    // lanes c = 13..15 read the zero padding columns (their sums are dropped)
#pragma unroll
    for (int m = 0; m < BS; ++m) bcol[m] = sB[m * RS + c];
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      const float4* row = reinterpret_cast<const float4*>(sA + r * RS);
      float2 v = acc[r];
#pragma unroll
      for (int m2 = 0; m2 < 7; ++m2) {
        float4 a2 = row[m2];  // elements 2*m2, 2*m2+1 (broadcast)
        v = cfma2(make_float2(a2.x, a2.y), bcol[2 * m2], v);
        if (2 * m2 + 1 < BS) v = cfma2(make_float2(a2.z, a2.w), bcol[2 * m2 + 1], v);
      }
      acc[r] = v;
    }
    __syncwarp();  // all lanes done with this stage before it is refilled
    stage ^= 1;
  }
  if (!ok) {
    // bounded drain of copies in flight, then report and leave
    for (int s = 0; s < 2; ++s)
      if ((pending >> s) & 1u) mbar_wait(&bar[s], (phase >> s) & 1u);
    if (lane == 0 && g.err) atomicExch(g.err, 1);
    return;
  }
  // the two groups meet
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, 16);
    acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, 16);
  }
  const int q = g.item_blk[item];
  if constexpr (EPI == EPI_STORE || EPI == EPI_ADD) {
    float2* __restrict__ C = static_cast<float2*>(g.C);
    if (h == 0 && c < BS) {
      if constexpr (EPI == EPI_ADD) {  // C += acc (all loads first)
        float2 old[BS];
#pragma unroll
        for (int r = 0; r < BS; ++r) old[r] = C[(int64_t)q * SB + r * RS + c];
#pragma unroll
        for (int r = 0; r < BS; ++r) acc[r] = make_float2(old[r].x + acc[r].x, old[r].y + acc[r].y);
      }
#pragma unroll
      for (int r = 0; r < BS; ++r) C[(int64_t)q * SB + r * RS + c] = acc[r];
    }
    // delta form: also W = K + M in FP32 (K in FP64, dense blocks, through
    // the map from this pattern to K's; -1 = no K block).  In the incremental
    // form this is the lo-part product and g.addend holds the hi part:
    // W = dK + (M_hi + M_lo), summed in FP64.
    if (g.base) {
      const double2* __restrict__ Kb = static_cast<const double2*>(g.base);
      const float2* __restrict__ Mh = static_cast<const float2*>(g.addend);
      float2* __restrict__ W = static_cast<float2*>(g.U);
      const int kq = g.add_map ? g.add_map[q] : q;
      if (h == 0 && c < BS) {
        double2 kv[BS];
        float2 mh[BS];
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          kv[r] = (kq >= 0) ? Kb[(int64_t)kq * NE + r * BS + c] : make_double2(0.0, 0.0);
          mh[r] = Mh ? Mh[(int64_t)q * SB + r * RS + c] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < BS; ++r)
          W[(int64_t)q * SB + r * RS + c] =
              make_float2((float)(((double)mh[r].x + (double)acc[r].x) + kv[r].x),
                          (float)(((double)mh[r].y + (double)acc[r].y) + kv[r].y));
      }
    }
  } else if constexpr (EPI == EPI_DELTA_SANDWICH) {
    // K'_ij = K_ij + M_ij + acc for j >= i (K in FP64, NE layout); mirror;
    // hermitian diagonal blocks
    const int i = g.rowidx[q], j = g.colidx[q];
    double2* __restrict__ K = static_cast<double2*>(g.C);
    const double2* __restrict__ base = static_cast<const double2*>(g.base);
    const float2* __restrict__ add = static_cast<const float2*>(g.addend);
    const int aq = g.add_map ? g.add_map[q] : q;
    double2 val[BS];
    if (h == 0 && c < BS) {
      // all loads first (K and its mirror may alias later stores)
      float2 mv[BS];
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        val[r] = base[(int64_t)q * NE + r * BS + c];
        mv[r] = (aq >= 0) ? add[(int64_t)aq * SB + r * RS + c] : make_float2(0.f, 0.f);
      }
      if (g.base2) {
        // incremental form: dK' = dK + R + M_hi + M_lo + N_lo + N_hi, every
        // part added in FP64 (the lo parts are below FP32 resolution of the hi)
        const double2* __restrict__ R = static_cast<const double2*>(g.base2);
        const float2* __restrict__ Nl = static_cast<const float2*>(g.addend2);
        const float2* __restrict__ Ml = static_cast<const float2*>(g.addend3);
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          double2 rv = R[(int64_t)q * NE + r * BS + c];
          float2 nl = Nl[(int64_t)q * SB + r * RS + c];
          float2 ml = (aq >= 0) ? Ml[(int64_t)aq * SB + r * RS + c] : make_float2(0.f, 0.f);
          val[r] = make_double2(val[r].x + rv.x + (((double)nl.x + (double)ml.x) + (double)acc[r].x),
                                val[r].y + rv.y + (((double)nl.y + (double)ml.y) + (double)acc[r].y));
          acc[r] = make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int r = 0; r < BS; ++r)
        val[r] = make_double2(val[r].x + ((double)mv[r].x + (double)acc[r].x),
                              val[r].y + ((double)mv[r].y + (double)acc[r].y));
    }
    if (i != j) {
      if (h == 0 && c < BS) {
        const int qt = g.tmap[q];
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          K[(int64_t)q * NE + r * BS + c] = val[r];
          K[(int64_t)qt * NE + c * BS + r] = make_double2(val[r].x, -val[r].y);
        }
      }
    } else {
      // pair (r,c) with (c,r) through shared memory (this warp's staging area;
      // every copy into it has completed)
      double2* sK = reinterpret_cast<double2*>(wsm);
      __syncwarp();
      if (h == 0 && c < BS) {
#pragma unroll
        for (int r = 0; r < BS; ++r) sK[r * BS + c] = val[r];
      }
      __syncwarp();
      double herm = 0.0;
      if (h == 0 && c < BS) {
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          double2 tv = sK[c * BS + r];
          double dr = val[r].x - tv.x, di = val[r].y + tv.y;
          herm = fmax(herm, sqrt(dr * dr + di * di));
          K[(int64_t)q * NE + r * BS + c] = make_double2(0.5 * (val[r].x + tv.x), 0.5 * (val[r].y - tv.y));
        }
      }
      for (int off = 16; off > 0; off >>= 1) herm = fmax(herm, __shfl_xor_sync(0xffffffffu, herm, off));
      if (lane == 0 && g.herm_max) amax_nonneg(g.herm_max, herm);
    }
  }
}

// ---------------------------------------------------------------------------
// real: 4 groups x 8 lanes, lane (h, cl) owns output columns 2cl and 2cl+1
// ---------------------------------------------------------------------------
template <int EPI>
__global__ void __launch_bounds__(WARPS * 32, 4) k_gemm13_r32(GemmArgs g) {
  constexpr int NT = 4;
  constexpr int WBUF = NT * Slot<float>::STRIDE;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int h = lane >> 3;
  const int cl = lane & 7;
  const int c0 = 2 * cl, c1 = 2 * cl + 1;
  const int64_t item = (int64_t)blockIdx.x * WARPS + warp;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  Smem* ctl = reinterpret_cast<Smem*>(dyn_smem);
  float* wsm = reinterpret_cast<float*>(dyn_smem + 128) + (size_t)warp * 2 * WBUF;
  if (item >= g.n_items) return;
  uint64_t* bar = ctl->bar[warp];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncwarp();

  const float* __restrict__ A = static_cast<const float*>(g.A);
  const float* __restrict__ B = static_cast<const float*>(g.B);
  const float* __restrict__ Z = static_cast<const float*>(g.zero);
  const int64_t t0 = g.ptr[item], t1 = g.ptr[item + 1];

  float acc0[BS], acc1[BS];
#pragma unroll
  for (int r = 0; r < BS; ++r) acc0[r] = acc1[r] = 0.f;

  unsigned phase = 0u;    // bit s: parity to wait for on stage s
  unsigned pending = 0u;  // bit s: copies in flight into stage s
  bool ok = true;
  int stage = 0;
  int nblk = -1;  // this lane's block index for the next group (prefetched)
  if (t0 < t1) {
    issue_group<float, NT>(wsm, A, B, group_block<NT>(g.ab, t0, t1, lane), Z, &bar[0], lane);
    nblk = group_block<NT>(g.ab, t0 + NT, t1, lane);
    pending |= 1u;
  }
  for (int64_t tb = t0; tb < t1; tb += NT) {
    if (tb + NT < t1) {
      issue_group<float, NT>(wsm + (stage ^ 1) * WBUF, A, B, nblk, Z, &bar[stage ^ 1], lane);
      nblk = group_block<NT>(g.ab, tb + 2 * NT, t1, lane);  // used one iteration later
      pending |= 1u << (stage ^ 1);
    }
    if (!mbar_wait(&bar[stage], (phase >> stage) & 1u)) {
      ok = false;
      break;
    }
    phase ^= 1u << stage;
    pending &= ~(1u << stage);
    const float* sA = wsm + stage * WBUF + h * Slot<float>::STRIDE;
    const float* sB = sA + SB;
    float b0[BS], b1[BS];
    // columns c0, c1 <= 15: the padding columns 13..15 hold zeros (sums dropped)
#pragma unroll
    for (int m = 0; m < BS; ++m) {
      float2 bb = *reinterpret_cast<const float2*>(sB + m * RS + c0);
      b0[m] = bb.x;
      b1[m] = bb.y;
    }
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      const float4* row = reinterpret_cast<const float4*>(sA + r * RS);
      float v0 = acc0[r], v1 = acc1[r];
#pragma unroll
      for (int m4 = 0; m4 < 4; ++m4) {
        float4 a4 = row[m4];
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int m = 4 * m4 + u;
          if (m < BS) {
            v0 = fmaf(av[u], b0[m], v0);
            v1 = fmaf(av[u], b1[m], v1);
          }
        }
      }
      acc0[r] = v0;
      acc1[r] = v1;
    }
    __syncwarp();
    stage ^= 1;
  }
  if (!ok) {
    for (int s = 0; s < 2; ++s)
      if ((pending >> s) & 1u) mbar_wait(&bar[s], (phase >> s) & 1u);
    if (lane == 0 && g.err) atomicExch(g.err, 1);
    return;
  }
#pragma unroll
  for (int r = 0; r < BS; ++r) {
    acc0[r] += __shfl_xor_sync(0xffffffffu, acc0[r], 8);
    acc0[r] += __shfl_xor_sync(0xffffffffu, acc0[r], 16);
    acc1[r] += __shfl_xor_sync(0xffffffffu, acc1[r], 8);
    acc1[r] += __shfl_xor_sync(0xffffffffu, acc1[r], 16);
  }
  if (h != 0 || c0 >= BS) return;
  const int q = g.item_blk[item];
  float* __restrict__ C = static_cast<float*>(g.C);
  if constexpr (EPI == EPI_STORE) {
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      if (c1 < BS) *reinterpret_cast<float2*>(&C[(int64_t)q * SB + r * RS + c0]) = make_float2(acc0[r], acc1[r]);
      else C[(int64_t)q * SB + r * RS + c0] = acc0[r];
    }
  } else if constexpr (EPI == EPI_STORE_ACC) {
    // U += coef * C (coef real or imaginary); every load is issued before the
    // first store so the read-modify-writes do not serialise on L2 round trips.
    // C is not stored when g.C is null (the last power is needed only in U).
    float2* __restrict__ U = static_cast<float2*>(g.U);
    const int uq = g.umap ? g.umap[q] : q;
    const float cf = (float)g.coef;
    if (uq >= 0) {
      float4 uv[BS];  // (U[r][c0], U[r][c1]) as 4 floats; c1 <= 13 stays inside the padded row
#pragma unroll
      for (int r = 0; r < BS; ++r) uv[r] = *reinterpret_cast<const float4*>(&U[(int64_t)uq * SB + r * RS + c0]);
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        if (g.coef_imag) {
          uv[r].y += cf * acc0[r];
          uv[r].w += cf * acc1[r];
        } else {
          uv[r].x += cf * acc0[r];
          uv[r].z += cf * acc1[r];
        }
      }
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        float2* dst = &U[(int64_t)uq * SB + r * RS + c0];
        if (c1 < BS) *reinterpret_cast<float4*>(dst) = uv[r];
        else *dst = make_float2(uv[r].x, uv[r].y);
      }
      // last power: U is complete; also write its conjugate transpose per block
      if (g.base) {
        float2* __restrict__ UH = static_cast<float2*>(const_cast<void*>(g.base));
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          UH[(int64_t)uq * SB + c0 * RS + r] = make_float2(uv[r].x, -uv[r].y);
          if (c1 < BS) UH[(int64_t)uq * SB + c1 * RS + r] = make_float2(uv[r].z, -uv[r].w);
        }
      }
    }
    if (C) {
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        if (c1 < BS) *reinterpret_cast<float2*>(&C[(int64_t)q * SB + r * RS + c0]) = make_float2(acc0[r], acc1[r]);
        else C[(int64_t)q * SB + r * RS + c0] = acc0[r];
      }
    }
  }
}

}  // namespace f32

// Launches the FP32 13-function kernels; false if the variant is not one of
// theirs.  B^dagger operands must be passed pre-transposed (b_dag = false).
bool launch_gemm13_f32(bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g, cudaStream_t st) {
  using namespace f32;
  if (a_dag || b_dag) return false;
  if (g.n_items == 0) return true;
  RT_REQUIRE(g.zero != nullptr, RT_EINTERNAL, "FP32 products need a zero block");
  int64_t grid = (g.n_items + WARPS - 1) / WARPS;
  RT_REQUIRE(grid < (1ll << 31), RT_EINTERNAL, "grid too large");
  const size_t smem_c = 128 + (size_t)WARPS * 2 * (2 * Slot<float2>::STRIDE) * sizeof(float2);  // 2 stages x NT=2
  const size_t smem_r = 128 + (size_t)WARPS * 2 * (4 * Slot<float>::STRIDE) * sizeof(float);    // 2 stages x NT=4
  static bool attr_done = false;
  if (!attr_done) {
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_c32<EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_c32<EPI_DELTA_SANDWICH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_c32<EPI_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_r32<EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_r32<EPI_STORE_ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    attr_done = true;
  }
  if (cplx) {
    if (epi == EPI_STORE) k_gemm13_c32<EPI_STORE><<<(unsigned)grid, WARPS * 32, smem_c, st>>>(g);
    else if (epi == EPI_ADD) k_gemm13_c32<EPI_ADD><<<(unsigned)grid, WARPS * 32, smem_c, st>>>(g);
    else if (epi == EPI_DELTA_SANDWICH) k_gemm13_c32<EPI_DELTA_SANDWICH><<<(unsigned)grid, WARPS * 32, smem_c, st>>>(g);
    else return false;
  } else {
    if (epi == EPI_STORE) k_gemm13_r32<EPI_STORE><<<(unsigned)grid, WARPS * 32, smem_r, st>>>(g);
    else if (epi == EPI_STORE_ACC) k_gemm13_r32<EPI_STORE_ACC><<<(unsigned)grid, WARPS * 32, smem_r, st>>>(g);
    else return false;
  }
  RT_CUDA_CHECK(cudaGetLastError());
  return true;
}

}  // namespace rt
