// FP32 block products for 13-function atoms (the mixed-precision path).
//
// Same contraction as spgemm.cu (C_ij = sum_k op(A)_ik op(B)_kj over the
// triple list of the output block, k ascending), laid out for FP32 throughput
// on the CUDA cores:
//   * FP32 matrices of 13-function atoms are stored with a padded row stride
//     of 16 (one block = 13 x 16 elements = 832 B real / 1664 B complex, 16 B
//     aligned), the same layout the blocks take in shared memory;
//   * one warp owns one 13x13 output block; one elected lane arms the stage's
//     mbarrier and lanes 0..2NT-1 stream the A and B blocks of the next NT
//     triples into shared memory with 1D TMA bulk copies (cp.async.bulk),
//     two stages per warp (the next group is in flight while the current one
//     is multiplied);
//   * the warp splits into NT lane groups, one staged triple each (complex:
//     2 groups of 16 lanes, 1 output column per lane; real: 4 groups of 8
//     lanes, each lane 7 rows x 4 columns); a lane keeps its B columns in
//     registers and reads the A rows as shared-memory broadcasts (one 16-byte
//     skew per slot puts the groups' broadcasts on different banks);
//   * the groups' partial sums meet in shared memory, and the epilogue walks
//     the block's 169 elements with all 32 lanes (FP64 K blocks are read and
//     written contiguously);
//   * B^dagger operands are pre-transposed (a conjugate-transposed copy of
//     U - I), so every staged block is a straight copy;
//   * every wait on an mbarrier is bounded in time (the launch's budget, 2 s
//     by default, read from the global timer): on expiry the kernel records an
//     error code, waits (bounded) for its copies in flight and returns.
#include <algorithm>

#include "rt_internal.cuh"
#include "rt_ptx.cuh"

namespace rt {

namespace f32 {

constexpr int BS = 13;
constexpr int NE = BS * BS;
constexpr int RS = 16;        // padded row stride
constexpr int SB = BS * RS;   // padded block (elements)
// Pipeline shape per kernel: warps per CTA and stages per warp (a stage holds
// NT staged triples; S stages keep S - 1 groups in flight while one is used).
constexpr int WARPS = 4;         // complex kernel
constexpr int C_STAGES = 2;
constexpr int R_WARPS = 4;       // real kernel
constexpr int R_STAGES = 2;
constexpr int MAX_STAGES = 4;
// One staged triple = A block + B block + 16 bytes of skew, so that the lane
// groups' broadcast reads of different triples fall on different banks.
template <typename V>
struct Slot {
  static constexpr int SKEW = 16 / sizeof(V);
  static constexpr int STRIDE = 2 * SB + SKEW;  // elements
};
constexpr long long DRAIN_NS = 2000000000ll;  // budget of the drain after a wait gave up (2 s)
// outcomes of a warp's main loop, also the values of the device error word
// (the word keeps the largest code any warp recorded)
constexpr int WAIT_OK = 0;
constexpr int WAIT_EXPIRED = 1;   // a wait gave up; every copy in flight was drained
constexpr int DRAIN_EXPIRED = 2;  // the drain gave up as well: copies may still have landed late

__device__ __forceinline__ float2 cfma2(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}

// Two FP32 values in one 64-bit register (low half first) and the packed
// arithmetic of sm_100+ on such pairs: one instruction, two roundings.
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(uint64_t v) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
  return f;
}
__device__ __forceinline__ uint64_t fma_x2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul_x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t add_x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub_x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ void amax_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Issue the TMA copies of one group of NT triples into `buf` (slot k holds A
// at k*STRIDE and B at k*STRIDE + SB).  Lane 0 arms the stage's mbarrier with
// the byte count; then lanes 0..2NT-1 issue one bulk copy each (all copies in
// one warp-wide instruction).  `blk` is the lane's block index for this group,
// loaded one group ahead (-1: past the end of the item: copy a zero block, so
// that every lane group multiplies without a branch).
template <typename V, int NT>
__device__ __forceinline__ void issue_group(V* buf, const V* __restrict__ A, const V* __restrict__ B, int blk,
                                            const V* __restrict__ zero, uint64_t* bar, int lane) {
  constexpr unsigned BYTES = SB * sizeof(V);
  if (lane == 0) mbar_expect_tx(bar, NT * 2u * BYTES);
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
  uint64_t bar[8][MAX_STAGES];  // [warp][stage]
};
static_assert(WARPS <= 8 && R_WARPS <= 8 && C_STAGES <= MAX_STAGES && R_STAGES <= MAX_STAGES, "pipeline shape");
static_assert(sizeof(Smem) <= 256, "control block");

// dynamic shared memory per CTA (control block + every warp's stages) and the
// CTAs per SM it leaves room for (227 KB per SM for CTAs)
// complex kernel with NS stages per warp (C_STAGES by default; the tuner also tries 3)
constexpr size_t smem_c(int ns) { return 256 + (size_t)WARPS * ns * (2 * Slot<float2>::STRIDE) * sizeof(float2); }
constexpr int minb_c(int ns) { return (int)((227 * 1024) / (smem_c(ns) + 1024)); }
constexpr size_t SMEM_C = smem_c(C_STAGES);  // NT = 2
constexpr size_t SMEM_R = 256 + (size_t)R_WARPS * R_STAGES * (4 * Slot<float>::STRIDE) * sizeof(float);  // NT = 4
constexpr int MINB_C = (int)((227 * 1024) / (SMEM_C + 1024));
constexpr int MINB_R = (int)((227 * 1024) / (SMEM_R + 1024));
static_assert(MINB_C >= 1 && MINB_R >= 1 && minb_c(3) >= 1, "stages do not fit in shared memory");

// Elements of a 13 x 13 block handled by one lane in the per-element epilogues.
constexpr int EPT = (NE + 31) / 32;

// ---------------------------------------------------------------------------
// Main loop shared by both kernels: stream the item's triples through the
// warp's S stages, NT triples per stage (lane group h takes slot h), S - 1
// groups in flight, and call `mac(sA, sB)` on each staged pair.  Returns
// WAIT_OK, WAIT_EXPIRED (a wait expired; the copies in flight were then
// drained) or DRAIN_EXPIRED (the drain ran out too: copies may still land).
// ---------------------------------------------------------------------------
template <typename V, int NT, int S, typename F>
__device__ __forceinline__ int stream_triples(V* wsm, uint64_t* bar, const V* __restrict__ A,
                                               const V* __restrict__ B, const V* __restrict__ Z,
                                               const int2* __restrict__ ab, int64_t t0, int64_t t1, int lane,
                                               int h, long long wait_ns, unsigned& phase, F&& mac) {
  // phase, bit s: parity to wait for on stage s (carried from item to item:
  // every stage's copies are waited for before an item ends)
  constexpr int WBUF = NT * Slot<V>::STRIDE;
  unsigned pending = 0u;  // bit s: copies in flight into stage s
  int64_t tnext = t0;     // first triple of the next group to issue
  int snext = 0;          // the stage it goes into
  int blk = group_block<NT>(ab, t0, t1, lane);  // this lane's block index for that group
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if (tnext < t1) {
      issue_group<V, NT>(wsm + snext * WBUF, A, B, blk, Z, &bar[snext], lane);
      pending |= 1u << snext;
      tnext += NT;
      snext = snext + 1 == S ? 0 : snext + 1;
      blk = group_block<NT>(ab, tnext, t1, lane);
    }
  }
  int stage = 0;
  for (int64_t tb = t0; tb < t1; tb += NT) {
    if (tnext < t1) {
      // refill the stage used in the previous iteration (released by its __syncwarp)
      issue_group<V, NT>(wsm + snext * WBUF, A, B, blk, Z, &bar[snext], lane);
      pending |= 1u << snext;
      tnext += NT;
      snext = snext + 1 == S ? 0 : snext + 1;
      blk = group_block<NT>(ab, tnext, t1, lane);  // used one iteration later
    }
    if (!mbar_wait(&bar[stage], (phase >> stage) & 1u, wait_ns)) {
      // bounded drain of every stage with copies in flight (this one included):
      // no copy may still be landing in shared memory when the warp leaves.
      // A drain that also runs out leaves copies in flight: reported apart.
      int code = WAIT_EXPIRED;
      for (int st = 0; st < S; ++st)
        if ((pending >> st) & 1u)
          if (!mbar_wait(&bar[st], (phase >> st) & 1u, DRAIN_NS)) code = DRAIN_EXPIRED;
      return code;
    }
    phase ^= 1u << stage;
    pending &= ~(1u << stage);
    const V* sA = wsm + stage * WBUF + h * Slot<V>::STRIDE;
    mac(sA, sA + SB);
    __syncwarp();  // all lanes done with this stage before it is refilled
    stage = stage + 1 == S ? 0 : stage + 1;
  }
  return WAIT_OK;
}

// ---------------------------------------------------------------------------
// complex: 2 lane groups x 16 lanes; lane (h, c) owns output column c of the
// triple in slot h (columns 13..15 are padding: zero B columns, sums
// dropped).  Partial sums meet in shared memory; the epilogue then walks the
// 169 elements of the block with all 32 lanes.
// ---------------------------------------------------------------------------
//
// PK = true: the packed variant.  A arrives column-planar (for each column m
// of the block: the real parts of rows 0..15, then the imaginary parts; rows
// 13..15 zero), so a column of A is a run of broadcast loads, and a lane
// (h, c) accumulates row pairs (2p, 2p+1) of its output column with one
// fma.rn.f32x2 per pair and partial product: per column m of A,
//   re += A_re(:,m) B_re(m,c),  re_n += A_im(:,m) B_im(m,c),
//   im += A_re(:,m) B_im(m,c) + A_im(:,m) B_re(m,c),
// and the running sum takes re - re_n and im once per triple.  B stays in
// the row layout; W (delta form) is written column-planar, since it is the A
// operand of the next product.
template <int EPI, bool PK, int NS>
__device__ __forceinline__ int c32_item(const GemmArgs& g, int64_t item, float2* wsm, uint64_t* bar,
                                        unsigned& phase, int lane, int h, int c, long long wait_ns) {
  constexpr int NT = 2;
  float2 acc[BS];
#pragma unroll
  for (int r = 0; r < BS; ++r) acc[r] = make_float2(0.f, 0.f);
  constexpr int NP = (BS + 1) / 2;  // row pairs (the last one holds padding row 13)
  uint64_t top_re[NP], top_im[NP];  // packed variant: running sums of row pairs
#pragma unroll
  for (int p = 0; p < NP; ++p) top_re[p] = top_im[p] = 0ull;

  int ok;
  if constexpr (PK) {
    ok = stream_triples<float2, NT, NS>(
        wsm, bar, static_cast<const float2*>(g.A), static_cast<const float2*>(g.B),
        static_cast<const float2*>(g.zero), g.ab, g.ptr[item], g.ptr[item + 1], lane, h, wait_ns, phase,
        [&](const float2* sA, const float2* sB) {
          const float* a = reinterpret_cast<const float*>(sA);
          uint64_t pre[NP], pren[NP], pim[NP];  // this triple's partial sums
#pragma unroll
          for (int m = 0; m < BS; ++m) {
            const float2 b = sB[m * RS + c];
            const uint64_t bxx = pk2(b.x, b.x), byy = pk2(b.y, b.y);
            const float* colm = a + m * 2 * RS;  // real parts of column m, then imaginary parts
            uint64_t ar[NP], ai[NP];
#pragma unroll
            for (int q4 = 0; q4 < 3; ++q4) {
              const float4 r4 = reinterpret_cast<const float4*>(colm)[q4];
              const float4 i4 = reinterpret_cast<const float4*>(colm + RS)[q4];
              ar[2 * q4] = pk2(r4.x, r4.y);
              ar[2 * q4 + 1] = pk2(r4.z, r4.w);
              ai[2 * q4] = pk2(i4.x, i4.y);
              ai[2 * q4 + 1] = pk2(i4.z, i4.w);
            }
            {
              const float2 r2 = reinterpret_cast<const float2*>(colm)[6];  // rows 12, 13
              const float2 i2 = reinterpret_cast<const float2*>(colm + RS)[6];
              ar[6] = pk2(r2.x, r2.y);
              ai[6] = pk2(i2.x, i2.y);
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              if (m == 0) {
                pre[p] = mul_x2(ar[p], bxx);
                pren[p] = mul_x2(ai[p], byy);
                pim[p] = fma_x2(ai[p], bxx, mul_x2(ar[p], byy));
              } else {
                pre[p] = fma_x2(ar[p], bxx, pre[p]);
                pren[p] = fma_x2(ai[p], byy, pren[p]);
                pim[p] = fma_x2(ar[p], byy, pim[p]);
                pim[p] = fma_x2(ai[p], bxx, pim[p]);
              }
            }
          }
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            top_re[p] = add_x2(top_re[p], sub_x2(pre[p], pren[p]));
            top_im[p] = add_x2(top_im[p], pim[p]);
          }
        });
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 re = upk2(top_re[p]), im = upk2(top_im[p]);
      acc[2 * p] = make_float2(re.x, im.x);
      if (2 * p + 1 < BS) acc[2 * p + 1] = make_float2(re.y, im.y);
    }
  } else {
  ok = stream_triples<float2, NT, NS>(
      wsm, bar, static_cast<const float2*>(g.A), static_cast<const float2*>(g.B),
      static_cast<const float2*>(g.zero), g.ab, g.ptr[item], g.ptr[item + 1], lane, h, wait_ns, phase,
      [&](const float2* sA, const float2* sB) {
        float2 bcol[BS];
#pragma unroll
        for (int m = 0; m < BS; ++m) bcol[m] = sB[m * RS + c];
#pragma unroll
        for (int r = 0; r < BS; ++r) {
          const float4* row = reinterpret_cast<const float4*>(sA + r * RS);
          // two-level sum: this triple's 13 terms in a fresh register, then
          // one addition into the running sum (the running sum takes one
          // rounding per triple instead of one per term)
          float2 v = make_float2(0.f, 0.f);
#pragma unroll
          for (int m2 = 0; m2 < 7; ++m2) {
            const float4 a2 = row[m2];  // A[r][2m2], A[r][2m2+1] (broadcast in the group)
            v = cfma2(make_float2(a2.x, a2.y), bcol[2 * m2], v);
            if (2 * m2 + 1 < BS) v = cfma2(make_float2(a2.z, a2.w), bcol[2 * m2 + 1], v);
          }
          acc[r].x += v.x;
          acc[r].y += v.y;
        }
      });
  }
  if (ok != WAIT_OK) return ok;
  // partial sums of the two groups to shared memory (every copy has landed)
  float2* part = wsm;  // [NT][BS][RS]
#pragma unroll
  for (int r = 0; r < BS; ++r) part[h * SB + r * RS + c] = acc[r];
  __syncwarp();
  float2 sum[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = lane + 32 * k;
    sum[k] = make_float2(0.f, 0.f);
    if (e < NE) {
      const int r = e / BS, c = e - BS * r;
#pragma unroll
      for (int hh = 0; hh < NT; ++hh) {
        const float2 v = part[hh * SB + r * RS + c];
        sum[k].x += v.x;
        sum[k].y += v.y;
      }
    }
  }
  const int q = g.item_blk[item];
  if constexpr (EPI == EPI_STORE || EPI == EPI_ADD) {
    float2* __restrict__ C = static_cast<float2*>(g.C);
    if constexpr (EPI == EPI_ADD) {  // C += acc (all loads first)
      float2 old[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        old[k] = e < NE ? C[(int64_t)q * SB + (e / BS) * RS + e % BS] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < EPT; ++k) sum[k] = make_float2(sum[k].x + old[k].x, sum[k].y + old[k].y);
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = lane + 32 * k;
      if (e < NE) C[(int64_t)q * SB + (e / BS) * RS + e % BS] = sum[k];
    }
    // delta form: also W = K + M in FP32 (K in FP64, dense blocks, through
    // the map from this pattern to K's; -1 = no K block); in the reference
    // split K is dK = K - K_ref
    if (g.base) {
      const double2* __restrict__ Kb = static_cast<const double2*>(g.base);
      float2* __restrict__ W = static_cast<float2*>(g.U);
      const int kq = g.add_map ? g.add_map[q] : q;
      double2 kv[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        kv[k] = make_double2(0.0, 0.0);
        if (e < NE && kq >= 0) kv[k] = Kb[(int64_t)kq * NE + e];
      }
      if constexpr (PK) {
        // column-planar W through shared memory (after the partial sums)
        float2* wt = part + NT * SB;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int e = lane + 32 * k;
          if (e < NE) wt[e] = make_float2((float)((double)sum[k].x + kv[k].x), (float)((double)sum[k].y + kv[k].y));
        }
        __syncwarp();
        float* __restrict__ Wp = reinterpret_cast<float*>(W) + (int64_t)q * (2 * SB);
        for (int idx = lane; idx < 2 * SB; idx += 32) {
          const int m = idx / (2 * RS), w = idx % (2 * RS), r = w % RS;
          float v = 0.f;
          if (r < BS) {
            const float2 t = wt[r * BS + m];
            v = w >= RS ? t.y : t.x;
          }
          Wp[idx] = v;
        }
      } else {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int e = lane + 32 * k;
          if (e < NE)
            W[(int64_t)q * SB + (e / BS) * RS + e % BS] =
                make_float2((float)((double)sum[k].x + kv[k].x), (float)((double)sum[k].y + kv[k].y));
        }
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
    double2 val[EPT];
    float2 mv[EPT];
    // all loads first (the stores of K below may alias them)
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = lane + 32 * k;
      val[k] = make_double2(0.0, 0.0);
      mv[k] = make_float2(0.f, 0.f);
      if (e < NE) {
        val[k] = base[(int64_t)q * NE + e];
        if (aq >= 0) mv[k] = add[(int64_t)aq * SB + (e / BS) * RS + e % BS];
      }
    }
    if (g.base2) {
      // reference split: dK' = dK + R + M + acc with R = U K_ref U^dagger - K_ref
      // (FP64, this output block)
      const double2* __restrict__ R = static_cast<const double2*>(g.base2);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        if (e < NE) {
          const double2 rv = R[(int64_t)q * NE + e];
          val[k] = make_double2(val[k].x + rv.x, val[k].y + rv.y);
        }
      }
    } else if (g.rpoly) {
      // the same R at this step's field, R(E) = sum_p E^p B_p, by Horner here;
      // coefficient by coefficient, so that the lane's loads of one B_p are
      // in flight together
      const double E = *g.poly_E;
      constexpr int HALF = (EPT + 1) / 2;  // elements per pass (register budget)
#pragma unroll
      for (int k0 = 0; k0 < EPT; k0 += HALF) {
        double2 rv[HALF];
        const double2* __restrict__ top = g.rpoly[g.rdeg];
#pragma unroll
        for (int k = 0; k < HALF; ++k) {
          const int e = lane + 32 * (k0 + k);
          rv[k] = (k0 + k < EPT && e < NE) ? top[(int64_t)q * NE + e] : make_double2(0.0, 0.0);
        }
        for (int p = g.rdeg - 1; p >= 0; --p) {
          const double2* __restrict__ cp = g.rpoly[p];
#pragma unroll
          for (int k = 0; k < HALF; ++k) {
            const int e = lane + 32 * (k0 + k);
            if (k0 + k < EPT && e < NE) {
              const double2 cv = cp[(int64_t)q * NE + e];
              rv[k] = make_double2(fma(rv[k].x, E, cv.x), fma(rv[k].y, E, cv.y));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < HALF; ++k)
          if (k0 + k < EPT) val[k0 + k] = make_double2(val[k0 + k].x + rv[k].x, val[k0 + k].y + rv[k].y);
      }
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      val[k] = make_double2(val[k].x + ((double)mv[k].x + (double)sum[k].x),
                            val[k].y + ((double)mv[k].y + (double)sum[k].y));
    if (i != j) {
      const int qt = g.tmap[q];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        if (e < NE) {
          const int r = e / BS, c = e - BS * r;
          K[(int64_t)q * NE + e] = val[k];
          K[(int64_t)qt * NE + c * BS + r] = make_double2(val[k].x, -val[k].y);
          if (g.kf32) {
            float2* __restrict__ Kf = static_cast<float2*>(g.kf32);
            Kf[(int64_t)q * SB + r * RS + c] = make_float2((float)val[k].x, (float)val[k].y);
            Kf[(int64_t)qt * SB + c * RS + r] = make_float2((float)val[k].x, (float)-val[k].y);
          }
        }
      }
    } else {
      // pair (r,c) with (c,r) through shared memory (after the partial sums)
      double2* sK = reinterpret_cast<double2*>(part + NT * SB);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        if (e < NE) sK[e] = val[k];
      }
      __syncwarp();
      double herm = 0.0;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        if (e < NE) {
          const int r = e / BS, c = e - BS * r;
          const double2 tv = sK[c * BS + r];
          const double dr = val[k].x - tv.x, di = val[k].y + tv.y;
          herm = fmax(herm, sqrt(dr * dr + di * di));
          const double2 w = make_double2(0.5 * (val[k].x + tv.x), 0.5 * (val[k].y - tv.y));
          K[(int64_t)q * NE + e] = w;
          if (g.kf32)
            static_cast<float2*>(g.kf32)[(int64_t)q * SB + r * RS + c] = make_float2((float)w.x, (float)w.y);
        }
      }
      for (int off = 16; off > 0; off >>= 1) herm = fmax(herm, __shfl_xor_sync(0xffffffffu, herm, off));
      if (lane == 0 && g.herm_max) amax_nonneg(g.herm_max, herm);
    }
  }
  return WAIT_OK;
}

// One warp per item (output block); a persistent launch (g.persistent) walks
// items with a grid-wide stride, and a grouped launch (g.grp) takes its items
// from several products at once: item i is item gitems[i].y of the product
// described by grp[gitems[i].x] (the same kernel and epilogue for all).
template <int EPI, bool PK, int NS>
__global__ void __launch_bounds__(WARPS * 32, minb_c(NS)) k_gemm13_c32(const __grid_constant__ GemmArgs g) {
  constexpr int NT = 2;
  constexpr int WBUF = NT * Slot<float2>::STRIDE;  // one stage of one warp (float2)
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int h = lane >> 4;
  const int c = lane & 15;
  int64_t item = (int64_t)blockIdx.x * WARPS + warp;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  Smem* ctl = reinterpret_cast<Smem*>(dyn_smem);
  float2* wsm = reinterpret_cast<float2*>(dyn_smem + 256) + (size_t)warp * NS * WBUF;
  if (item >= g.n_items) return;  // whole warp leaves together
  uint64_t* bar = ctl->bar[warp];
  if (lane == 0) {
    for (int st = 0; st < NS; ++st) mbar_init(&bar[st], 1);
    fence_mbar_init();
  }
  __syncwarp();
  const int64_t stride = g.persistent ? (int64_t)gridDim.x * WARPS : g.n_items;
  unsigned phase = 0u;
  for (bool first = true; item < g.n_items; item += stride, first = false) {
    if (!first) {
      // the last epilogue wrote this warp's buffers through the generic proxy;
      // order those writes before the next item's bulk copies land there
      fence_proxy_async_smem();
      __syncwarp();
    }
    const int2 gi = g.grp ? g.gitems[item] : make_int2(0, 0);
    const int ok = c32_item<EPI, PK, NS>(g.grp ? g.grp[gi.x] : g, g.grp ? (int64_t)gi.y : item, wsm, bar, phase,
                                         lane, h, c, g.wait_ns);
    if (ok != WAIT_OK) {
      if (lane == 0 && g.err) atomicMax(g.err, ok);
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// real: 4 lane groups x 2 row halves x 4 lanes; lane (h, half, cl) owns
// output rows 7 half .. 7 half + 6 and columns 4cl..4cl+3 of the triple in
// slot h (the second half's seventh row would be row 13: it multiplies the
// first row of the staged B block and is dropped).  Same staging and
// epilogue scheme as above.
// ---------------------------------------------------------------------------
template <int EPI>
__global__ void __launch_bounds__(R_WARPS * 32, MINB_R) k_gemm13_r32(GemmArgs g) {
  constexpr int NT = 4;
  constexpr int RH = 7;  // rows per half
  constexpr int WBUF = NT * Slot<float>::STRIDE;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int h = lane >> 3;
  const int half = (lane >> 2) & 1;
  const int cl = lane & 3;
  const int r0 = RH * half;
  const int64_t item = (int64_t)blockIdx.x * R_WARPS + warp;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  Smem* ctl = reinterpret_cast<Smem*>(dyn_smem);
  float* wsm = reinterpret_cast<float*>(dyn_smem + 256) + (size_t)warp * R_STAGES * WBUF;
  if (item >= g.n_items) return;
  uint64_t* bar = ctl->bar[warp];
  if (lane == 0) {
    for (int st = 0; st < R_STAGES; ++st) mbar_init(&bar[st], 1);
    fence_mbar_init();
  }
  __syncwarp();

  float4 acc[RH];
#pragma unroll
  for (int rr = 0; rr < RH; ++rr) acc[rr] = make_float4(0.f, 0.f, 0.f, 0.f);

  unsigned phase = 0u;
  const int ok = stream_triples<float, NT, R_STAGES>(
      wsm, bar, static_cast<const float*>(g.A), static_cast<const float*>(g.B), static_cast<const float*>(g.zero),
      g.ab, g.ptr[item], g.ptr[item + 1], lane, h, g.wait_ns, phase, [&](const float* sA, const float* sB) {
        float4 b[BS];  // B[m][4cl .. 4cl+3]
#pragma unroll
        for (int m = 0; m < BS; ++m) b[m] = *reinterpret_cast<const float4*>(sB + m * RS + 4 * cl);
#pragma unroll
        for (int rr = 0; rr < RH; ++rr) {
          const float4* row = reinterpret_cast<const float4*>(sA + (r0 + rr) * RS);
          float4 v = acc[rr];
#pragma unroll
          for (int m4 = 0; m4 < 4; ++m4) {
            const float4 a4 = row[m4];  // A[r][4m4 .. 4m4+3] (broadcast in the half group)
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int m = 4 * m4 + u;
              if (m < BS) {
                v.x = fmaf(av[u], b[m].x, v.x);
                v.y = fmaf(av[u], b[m].y, v.y);
                v.z = fmaf(av[u], b[m].z, v.z);
                v.w = fmaf(av[u], b[m].w, v.w);
              }
            }
          }
          acc[rr] = v;
        }
      });
  if (ok != WAIT_OK) {
    if (lane == 0 && g.err) atomicMax(g.err, ok);
    return;
  }
  float* part = wsm;  // [NT][BS][RS]
#pragma unroll
  for (int rr = 0; rr < RH; ++rr)
    if (r0 + rr < BS) *reinterpret_cast<float4*>(part + h * SB + (r0 + rr) * RS + 4 * cl) = acc[rr];
  __syncwarp();
  float sum[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = lane + 32 * k;
    sum[k] = 0.f;
    if (e < NE) {
      const int r = e / BS, c = e - BS * r;
#pragma unroll
      for (int hh = 0; hh < NT; ++hh) sum[k] += part[hh * SB + r * RS + c];
    }
  }
  const int q = g.item_blk[item];
  float* __restrict__ C = static_cast<float*>(g.C);
  if constexpr (EPI == EPI_STORE) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = lane + 32 * k;
      if (e < NE) C[(int64_t)q * SB + (e / BS) * RS + e % BS] = sum[k];
    }
  } else if constexpr (EPI == EPI_STORE_ACC) {
    // U += coef * C (coef real or imaginary), every load before the first
    // store; C is not stored when g.C is null (the last power is needed only
    // in U), and the last power also writes U^dagger per block (g.base).
    float2* __restrict__ U = static_cast<float2*>(g.U);
    const int uq = g.umap ? g.umap[q] : q;
    const float cf = (float)g.coef;
    if (uq >= 0) {
      float2 uv[EPT];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        uv[k] = e < NE ? U[(int64_t)uq * SB + (e / BS) * RS + e % BS] : make_float2(0.f, 0.f);
      }
      float2* __restrict__ UH = g.base ? static_cast<float2*>(const_cast<void*>(g.base)) : nullptr;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        if (e < NE) {
          const int r = e / BS, c = e - BS * r;
          if (g.coef_imag) uv[k].y += cf * sum[k];
          else uv[k].x += cf * sum[k];
          U[(int64_t)uq * SB + r * RS + c] = uv[k];
          if (UH) UH[(int64_t)uq * SB + c * RS + r] = make_float2(uv[k].x, -uv[k].y);
        }
      }
    }
    if (C) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = lane + 32 * k;
        if (e < NE) C[(int64_t)q * SB + (e / BS) * RS + e % BS] = sum[k];
      }
    }
  }
}

// One complex launch: NS stages per warp; a persistent launch runs at most
// as many CTAs as are resident at once (SMs x CTAs per SM).
template <int EPI, bool PK, int NS>
void launch_c32(const GemmArgs& g, cudaStream_t st) {
  constexpr size_t sm = smem_c(NS);
  static bool attr_done = false;
  if (!attr_done) {
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_c32<EPI, PK, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr_done = true;
  }
  int64_t grid = (g.n_items + WARPS - 1) / WARPS;
  if (g.persistent) {
    int dev = 0, sms = 0;
    RT_CUDA_CHECK(cudaGetDevice(&dev));
    RT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grid = std::min<int64_t>(grid, (int64_t)sms * minb_c(NS));
  }
  RT_REQUIRE(grid < (1ll << 31), RT_EINTERNAL, "grid too large");
  k_gemm13_c32<EPI, PK, NS><<<(unsigned)grid, WARPS * 32, sm, st>>>(g);
}

template <int EPI, bool PK>
void launch_c32_ns(const GemmArgs& g, cudaStream_t st) {
  if (g.stages == 3) launch_c32<EPI, PK, 3>(g, st);
  else launch_c32<EPI, PK, C_STAGES>(g, st);
}

}  // namespace f32

// Launches the FP32 13-function kernels; false if the variant is not one of
// theirs.  B^dagger operands must be passed pre-transposed (b_dag = false).
bool launch_gemm13_f32(bool cplx, bool a_dag, bool b_dag, Epilogue epi, const GemmArgs& g, cudaStream_t st) {
  using namespace f32;
  RT_REQUIRE(!g.a_planar || (cplx && !a_dag && !b_dag), RT_EINTERNAL,
             "column-planar A only for complex products with untransposed operands");
  RT_REQUIRE(g.stages == 0 || g.stages == C_STAGES || g.stages == 3, RT_EINTERNAL, "stages per warp: 2 or 3");
  RT_REQUIRE(!(g.grp || g.persistent || g.stages) || cplx, RT_EINTERNAL,
             "grouped, persistent and staged variants are complex-product launches");
  if (a_dag || b_dag) return false;
  if (g.n_items == 0) return true;
  RT_REQUIRE(g.zero != nullptr, RT_EINTERNAL, "FP32 products need a zero block");
  const int64_t grid_r = (g.n_items + R_WARPS - 1) / R_WARPS;
  const size_t smem_r = SMEM_R;
  static bool attr_done = false;
  if (!attr_done) {
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_r32<EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    RT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm13_r32<EPI_STORE_ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    attr_done = true;
  }
  if (cplx && g.a_planar) {
    if (epi == EPI_STORE) launch_c32_ns<EPI_STORE, true>(g, st);
    else if (epi == EPI_DELTA_SANDWICH) launch_c32_ns<EPI_DELTA_SANDWICH, true>(g, st);
    else RT_REQUIRE(false, RT_EINTERNAL, "column-planar A only with the store and delta-sandwich epilogues");
  } else if (cplx) {
    if (epi == EPI_STORE) launch_c32_ns<EPI_STORE, false>(g, st);
    else if (epi == EPI_ADD && !g.grp && !g.persistent && !g.stages) launch_c32<EPI_ADD, false, C_STAGES>(g, st);
    else if (epi == EPI_DELTA_SANDWICH) launch_c32_ns<EPI_DELTA_SANDWICH, false>(g, st);
    else return false;
  } else {
    RT_REQUIRE(grid_r < (1ll << 31), RT_EINTERNAL, "grid too large");
    if (epi == EPI_STORE) k_gemm13_r32<EPI_STORE><<<(unsigned)grid_r, R_WARPS * 32, smem_r, st>>>(g);
    else if (epi == EPI_STORE_ACC) k_gemm13_r32<EPI_STORE_ACC><<<(unsigned)grid_r, R_WARPS * 32, smem_r, st>>>(g);
    else return false;
  }
  RT_CUDA_CHECK(cudaGetLastError());
  return true;
}

}  // namespace rt
