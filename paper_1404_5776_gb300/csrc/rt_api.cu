// C ABI and step orchestration of the GB300 density-matrix RT-TDDFT library.
//
// One time step (paper Sec. II.A, eq. EM, eq. matrix_exp, Sec. V.A):
//   EM:  H(t+dt/2) = H0 - E D_j;  T = cut_{r_T}(S^-1 H);  T^n = cut_{r_U}(T T^{n-1});
//        U = sum_{n<6} (-i dt)^n T^n / n!
//   CN:  A = S + i dt/2 H, X <- X(2I - A X) (warm start), U = cut_{r_U}(X (S - i dt/2 H))
//   ETRS: U = cut_{r_U}(exp(-i dt/2 T(t+dt)) exp(-i dt/2 T(t)))
//   M4:  Om = -i dt/2 (T1 + T2) - sqrt(3) dt^2/12 [T2, T1] at the Gauss-Legendre
//        times t1, t2;  U = sum_{n<6} Om^n / n!  (powers cut to r_U)
//   M = cut_{r_M}(U K);  K' = M U^dagger on the upper blocks of P_K, mirrored;
//   Tr(K S), Tr(K D_xyz) recorded per step.
// All work runs on an internal stream ordered against the caller's stream with
// events; a step is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <tuple>

#include "rt_elementwise.cuh"
#include "rt_internal.cuh"

namespace rt {

// true multiply-adds of a triple list (block sizes without padding)
int64_t triple_true_macs(const Triples& T, const Pattern& A, bool a_dag, const Pattern& C, const int32_t* bsize,
                         Arena& arena, cudaStream_t st);

enum ProfClass { PC_FIELD = 0, PC_T, PC_TAYLOR, PC_UK, PC_MUDAG, PC_CN_HOT, PC_CN_U, PC_OBS, PC_MISC, PC_POLY, PC_N };
static const char* kProfNames[PC_N] = {"field_update", "gemm_T=SinvH",  "gemm_taylor_powers",
                                       "gemm_M=UK",    "gemm_K=MUdag",  "gemm_cn_hotelling",
                                       "gemm_cn_U=XB", "traces",        "misc",
                                       "field_polynomial_U"};

struct TripleKey {
  const Pattern *A, *B, *C;
  bool ad, bd, up;
  bool operator<(const TripleKey& o) const {
    return std::tie(A, B, C, ad, bd, up) < std::tie(o.A, o.B, o.C, o.ad, o.bd, o.up);
  }
};

struct TripleInfo {
  Triples t;
  TileList tiles;  // row tiles for the tensor-core kernel (built for the sandwich's FP32 13-function products)
  int64_t true_macs = 0;
  int64_t nnzb_a = 0, nnzb_b = 0;
  int64_t true_elems_a = 0, true_elems_b = 0, true_elems_c = 0;
};

struct Sys {
  int n_atoms = 0, B = 0;
  int64_t n_true = 0;
  std::vector<int32_t> bsize;
  int32_t* d_bsize = nullptr;
  double* d_pos = nullptr;
  bool periodic = false;
  double cell[3] = {0, 0, 0};
  double r_S = 0, r_H = 0;
  std::vector<double> h_pos;
  // patterns (owned by the context cache; several names may share one)
  Pattern *pS = nullptr, *pH = nullptr, *pSinv = nullptr, *pT = nullptr, *pU = nullptr, *pK = nullptr,
          *pM = nullptr, *pA = nullptr, *pW = nullptr;
  std::map<double, std::unique_ptr<Pattern>> pcache;
  std::unique_ptr<Pattern> pS_given, pH_given;
  std::map<TripleKey, std::unique_ptr<TripleInfo>> tcache;
  // FP64 values (padded blocks)
  double *S = nullptr, *H0 = nullptr, *D[3] = {nullptr, nullptr, nullptr}, *Hm = nullptr;
  double *Sinv = nullptr, *Zs = nullptr, *Xs2 = nullptr;
  double *T = nullptr, *P0 = nullptr, *P1 = nullptr, *T0 = nullptr, *TD = nullptr, *T2 = nullptr;
  // field polynomial of the EM propagator: U(E) = sum_m E^m V[m]
  std::vector<double2*> V;
  double* TDn = nullptr;        // -cut(S^-1 D)
  double2 *U = nullptr, *M = nullptr;
  std::vector<double2*> K;
  double2 *Acn = nullptr, *Bcn = nullptr, *X = nullptr, *Xn = nullptr, *Zc = nullptr;
  double2 *Sc = nullptr, *W = nullptr, *E = nullptr;
  // FP32 buffers (mixed precision)
  float *Tf = nullptr, *Pf0 = nullptr, *Pf1 = nullptr;
  float2 *dUf = nullptr, *dUH = nullptr, *Kf = nullptr, *Mf = nullptr, *Wf = nullptr;
  // FP32 ETRS: the two half-step differences exp(-i dt/2 T) - I; FP32 M4:
  // the powers of Om (dUa, dUb), Om itself and T2 in FP32
  float2 *dUa = nullptr, *dUb = nullptr, *Omf = nullptr;
  float* Tf2 = nullptr;
  // FP32 Hotelling iterations of the mixed CN step: A on P_A, X, Y = A X (then 2I - A X), X Y on P_U
  float2 *Acn32 = nullptr, *X32 = nullptr, *Y32 = nullptr, *Xn32 = nullptr;
  // reference split (FP32): K = K_ref + dK[kick] with one K_ref per system (the kicks of a
  // system stay O(kappa) apart), R = sym(cut(cut(U K_ref) U^dagger)) - K_ref in FP64
  // (constant U: R formed once; field polynomial: R(E) = sum_p E^p Bp[p] formed per step)
  double2 *Kref = nullptr, *Rm = nullptr;
  double* tref = nullptr;         // traces of K_ref (8 doubles)
  std::vector<double2*> dK;       // per kick
  std::vector<char> dk_fresh;     // per kick: dK holds K - K_ref (K itself is stale)
  bool ref_ready = false;         // K_ref and its traces are formed
  bool r_ready = false;           // R (constant U) or the Bp (field polynomial) match K_ref and U
  std::vector<double2*> Bp;       // coefficients of R(E) on P_K (Bp[0] includes -K_ref)
  double2** d_bp = nullptr;       // device table of the Bp (the K' epilogue evaluates R(E) from them)
  std::vector<float2*> V32;       // reference split: FP32 copies of V_1..V_deg (V32[0] null), the FP32 tail
                                  // of the per-step Horner pass for U(E) - I
  float2 *dUr = nullptr, *dUHr = nullptr;  // U - I stochastically rounded to FP32, and its block dagger
  bool u64_stale = false;         // the FP64 U is not formed per step (field polynomial, reference split)
  bool planar = false;            // dUr and Wf column-planar: the packed-FMA products of the reference split
  std::vector<float2*> Kfk;       // reference split, per kick: dK rounded to FP32 (kick 0 shares Kf); the
                                  // delta-sandwich epilogue rewrites it with every step
  std::vector<float2*> Mfk, Wfk;  // reference split, per kick: M and W = dK + M (kick 0 shares Mf, Wf)
  // maps
  int32_t *u_to_t = nullptr, *a_to_s = nullptr, *a_to_h = nullptr, *k_to_sT = nullptr, *k_to_hT = nullptr;
  int32_t *u_to_sinv = nullptr, *k_to_sinv = nullptr, *u_to_s = nullptr, *k_to_m = nullptr, *m_to_k = nullptr;
  // reductions
  double* red_items = nullptr;
  int64_t red_items_n = 0;
  double* red_part = nullptr;
  double* scal = nullptr;  // device scalars [16]
  double* rows_tmp = nullptr;
  bool sinv_ready = false;
  bool u_ready = false;
  bool duf_current = false;  // U - I in FP32 holds the last propagator (FP32 EM, ETRS, M4: U itself is not formed)
  int sinv_iters = 0;
  double sinv_resid = 0.0;
  std::string sinv_status;
};

// Grouped products of the reference split (one launch per product and block
// size across all (system, kick) pairs) and their launch shapes
constexpr int RT_N_STAGES = 4;  // 13-function M, 13-function K', 4-function M, 4-function K'
inline int stage_of(int B, bool kstage) { return (B == 13 ? 0 : 2) + (kstage ? 1 : 0); }
struct LaunchShape {
  int stages = 0;      // 13-function kernel: stages per warp (0 = 2)
  int persistent = 0;  // one resident wave of CTAs walking the items
};
struct StageGroup {
  GemmArgs* d_args = nullptr;  // device table: one entry per (system, kick) pair
  int2* d_items = nullptr;     // (pair, item) of every item, largest pairs first
  GemmArgs single{};           // the one pair's arguments (a stage with one pair launches without tables)
  std::vector<GemmArgs> host;  // host copy of the table (the tuner redirects the K' outputs)
  size_t out_bytes = 0, kf_bytes = 0;  // largest K' output and FP32 copy of one pair
  int64_t n_items = 0;
  int n_groups = 0;
  int B = 0;
  int planar = 0;
  bool bdag = false;
  double flops = 0, bytes = 0;
};

}  // namespace rt

struct rt_ctx {
  rt_params p{};
  rt::Allocator alloc;
  rt::Arena arena;
  cudaStream_t user = nullptr;
  cudaStream_t ws = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<std::unique_ptr<rt::Sys>> sys;
  rt::FieldParams field;
  rt::DevState* dstate = nullptr;
  void* zero32 = nullptr;  // one zero FP32 complex block (padded layout)
  int* d_err = nullptr;    // device error word of bounded waits
  long long wait_ns = 2000000000ll;  // budget of one bounded device wait
  uint32_t inject = 0;     // armed host-side fault injections (RT_FAULT_*)
  double* ring = nullptr;  // [capacity][n_slots][RT_NOBS]
  int n_slots = 0;
  int64_t host_step = 0;  // steps enqueued since the last time reset
  std::vector<int64_t> read_upto;  // per slot: steps already returned
  double t_host = 0.0;
  // graph
  cudaGraphExec_t gexec = nullptr;
  bool graph_dirty = true;
  // profiling / counting
  bool profiling = false;
  bool counting = false;
  double count_flops = 0.0, count_bytes = 0.0;
  int64_t count_kernels = 0;
  struct Prof {
    int64_t launches = 0;
    double ms = 0, flops = 0, bytes = 0;
  } prof[rt::PC_N];
  struct PendingEv {
    cudaEvent_t a, b;
    int cls;
    double flops, bytes;
  };
  std::vector<PendingEv> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
  // grouped products and the launch shapes the tuner chose
  rt::LaunchShape shape[rt::RT_N_STAGES];
  rt::StageGroup groups[rt::RT_N_STAGES];
  bool groups_built = false;
  // grouped traces of every (system, kick) pair (reference split, several pairs)
  rt::TracePair* d_tpairs = nullptr;
  double* tpart = nullptr;
  int n_tpairs = 0, tnb = 0;
  double tbytes = 0.0;
  bool poisoned = false;
  bool unrecoverable = false;  // a drain of copies in flight gave up: shared memory may have been written late
  std::string err;
};

static void check_device_error(rt_ctx* c);

namespace rt {

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------
template <class F>
static void run(rt_ctx* c, int cls, double flops, double bytes, F&& f, int kernels = 1) {
  if (c->counting) {
    c->count_flops += flops;
    c->count_bytes += bytes;
    c->count_kernels += kernels;
    return;
  }
  if (c->profiling) {
    std::pair<cudaEvent_t, cudaEvent_t> ev;
    if (!c->ev_free.empty()) {
      ev = c->ev_free.back();
      c->ev_free.pop_back();
    } else {
      RT_CUDA_CHECK(cudaEventCreate(&ev.first));
      RT_CUDA_CHECK(cudaEventCreate(&ev.second));
    }
    RT_CUDA_CHECK(cudaEventRecord(ev.first, c->ws));
    f();
    RT_CUDA_CHECK(cudaEventRecord(ev.second, c->ws));
    c->pending.push_back({ev.first, ev.second, cls, flops, bytes});
  } else {
    f();
  }
}

static void collect_profile(rt_ctx* c) {
  if (c->pending.empty()) return;
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
  for (auto& pe : c->pending) {
    float ms = 0.f;
    RT_CUDA_CHECK(cudaEventElapsedTime(&ms, pe.a, pe.b));
    auto& pr = c->prof[pe.cls];
    pr.launches += 1;
    pr.ms += ms;
    pr.flops += pe.flops;
    pr.bytes += pe.bytes;
    c->ev_free.push_back({pe.a, pe.b});
  }
  c->pending.clear();
}

static Pattern* pattern_for(rt_ctx* c, Sys& s, double r) {
  auto it = s.pcache.find(r);
  if (it != s.pcache.end()) return it->second.get();
  auto P = std::make_unique<Pattern>();
  build_pattern(*P, s.n_atoms, s.d_pos, s.periodic ? s.cell : nullptr, r, c->arena, c->ws);
  Pattern* raw = P.get();
  s.pcache[r] = std::move(P);
  return raw;
}

static TripleInfo& triples_for(rt_ctx* c, Sys& s, Pattern* A, bool ad, Pattern* B, bool bd, Pattern* C, bool up) {
  TripleKey key{A, B, C, ad, bd, up};
  auto it = s.tcache.find(key);
  if (it != s.tcache.end()) return *it->second;
  auto ti = std::make_unique<TripleInfo>();
  build_triples(ti->t, *A, ad, *B, bd, *C, up, c->arena, c->ws);
  ti->true_macs = triple_true_macs(ti->t, *A, ad, *C, s.d_bsize, c->arena, c->ws);
  ti->nnzb_a = A->nnzb;
  ti->nnzb_b = B->nnzb;
  auto elems = [&](const Pattern* P) {
    int64_t n = 0;
    for (int i = 0; i < s.n_atoms; ++i)
      for (int q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) n += (int64_t)s.bsize[i] * s.bsize[P->h_col[q]];
    return n;
  };
  ti->true_elems_a = elems(A);
  ti->true_elems_b = elems(B);
  {
    std::vector<int32_t> items(ti->t.n_items);
    if (ti->t.n_items)
      RT_CUDA_CHECK(cudaMemcpyAsync(items.data(), ti->t.item_blk, sizeof(int32_t) * ti->t.n_items,
                                    cudaMemcpyDeviceToHost, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    std::vector<int32_t> rowof(C->nnzb);
    for (int i = 0; i < s.n_atoms; ++i)
      for (int q = C->h_rowptr[i]; q < C->h_rowptr[i + 1]; ++q) rowof[q] = i;
    int64_t n = 0;
    for (int32_t q : items) n += (int64_t)s.bsize[rowof[q]] * s.bsize[C->h_col[q]];
    ti->true_elems_c = n;
  }
  if (ti->t.n_items > s.red_items_n) {
    s.red_items = c->arena.get_n<double>(ti->t.n_items);
    s.red_items_n = ti->t.n_items;
  }
  TripleInfo& ref = *ti;
  s.tcache[key] = std::move(ti);
  return ref;
}

static size_t nvals(const Sys& s, const Pattern* P) { return (size_t)P->nnzb * s.B * s.B; }
static bool incremental(const rt_ctx* c) { return c->p.incremental != 0; }
// elements of an FP32 matrix (13-function blocks padded to 13 x 16)
static size_t nvals32(const Sys& s, const Pattern* P) { return (size_t)P->nnzb * sb32(s.B); }

static int32_t* block_map(rt_ctx* c, const Pattern* src, const Pattern* dst, bool transpose) {
  int32_t* m = c->arena.get_n<int32_t>(src->nnzb);
  if (transpose) build_transpose_map(m, *src, *dst, c->ws);
  else build_block_map(m, *src, *dst, c->ws);
  return m;
}

// algorithmic flops / bytes of a product (true block sizes): every block of
// A and B read once, every output block written once
static double gemm_flops(const TripleInfo& ti, bool cplx) { return (cplx ? 8.0 : 2.0) * (double)ti.true_macs; }
static double gemm_bytes(const Sys&, const TripleInfo& ti, bool cplx, bool fp32) {
  double bpe = (cplx ? 2.0 : 1.0) * (fp32 ? 4.0 : 8.0);
  return bpe * (double)(ti.true_elems_a + ti.true_elems_b + ti.true_elems_c);
}

// The arguments of one block product, completed from its triple list and
// output pattern, with the overlap checks of its buffers.
static GemmArgs prepared(rt_ctx* c, Sys& s, TripleInfo& ti, bool fp32, bool cplx, Epilogue epi, GemmArgs g,
                         const Pattern* C) {
  g.item_blk = ti.t.item_blk;
  g.ptr = ti.t.ptr;
  g.ab = ti.t.ab;
  g.n_items = ti.t.n_items;
  g.tri = &ti.t;
  if (C) {
    g.rowidx = C->rowidx;
    g.colidx = C->col;
    g.tmap = C->tmap;
  }
  g.bsize = s.d_bsize;
  g.zero = c->zero32;
  g.err = c->d_err;
  g.wait_ns = c->wait_ns;
  // each output block is written by the one item that owns it while every
  // item reads the operands: an output or accumulator overlapping an operand
  // (the same buffer or any part of it) races
  {
    const size_t vbytes = (cplx ? 2 : 1) * (fp32 ? 4 : 8);
    const size_t op_blk = (size_t)(fp32 ? sb32(s.B) : s.B * s.B) * vbytes;
    const size_t out_blk = epi == EPI_DELTA_SANDWICH ? (size_t)s.B * s.B * 16 : op_blk;
    const size_t acc_blk = (size_t)(fp32 ? sb32(s.B) * 8 : s.B * s.B * 16);
    auto overlaps = [](const void* p, size_t np, const void* q, size_t nq) {
      const char *a = (const char*)p, *b = (const char*)q;
      return p && q && a < b + nq && b < a + np;
    };
    const size_t nA = (size_t)ti.nnzb_a * op_blk, nB = (size_t)ti.nnzb_b * op_blk;
    const size_t nC = C ? (size_t)C->nnzb * out_blk : 1;
    const size_t nU = (C && !g.umap) ? (size_t)C->nnzb * acc_blk : 1;
    RT_REQUIRE(!overlaps(g.C, nC, g.A, nA) && !overlaps(g.C, nC, g.B, nB), RT_EINTERNAL,
               "block product output overlaps an operand");
    RT_REQUIRE(!overlaps(g.U, nU, g.A, nA) && !overlaps(g.U, nU, g.B, nB), RT_EINTERNAL,
               "block product accumulator overlaps an operand");
    const size_t nF = C ? (size_t)C->nnzb * sb32(s.B) * 8 : 1;
    RT_REQUIRE(!overlaps(g.kf32, nF, g.A, nA) && !overlaps(g.kf32, nF, g.B, nB), RT_EINTERNAL,
               "FP32 copy of the output overlaps an operand");
  }
  return g;
}

static void gemm(rt_ctx* c, Sys& s, int cls, TripleInfo& ti, bool fp32, bool cplx, bool ad, bool bd, Epilogue epi,
                 GemmArgs g, const Pattern* C) {
  g = prepared(c, s, ti, fp32, cplx, epi, g, C);
  int B = s.B;
  RT_REQUIRE(!g.a_planar || (fp32 && cplx && B == 13 && !ti.tiles.built), RT_EINTERNAL,
             "column-planar operands belong to the packed CUDA-core products");
  RT_REQUIRE(!g.kf32 || (fp32 && cplx && epi == EPI_DELTA_SANDWICH && !ti.tiles.built), RT_EINTERNAL,
             "the FP32 copy of K' comes from the CUDA-core delta sandwich");
  if (fp32 && cplx && B == 13 && !ad && !bd && ti.tiles.built && (epi == EPI_STORE || epi == EPI_DELTA_SANDWICH)) {
    g.tl_n = ti.tiles.n_tiles;
    g.tl_item0 = ti.tiles.item0;
    g.tl_nitem = ti.tiles.nitem;
    g.tl_uptr = ti.tiles.uptr;
    g.tl_ua = ti.tiles.ua;
    g.tl_ub = ti.tiles.ub;
    run(c, cls, gemm_flops(ti, cplx), gemm_bytes(s, ti, cplx, fp32), [&] { launch_gemm13_tc(epi, g, c->ws); });
    return;
  }
  run(c, cls, gemm_flops(ti, cplx), gemm_bytes(s, ti, cplx, fp32),
      [&] { launch_gemm(B, fp32, cplx, ad, bd, epi, g, c->ws); });
}

// Device memory needed only inside one set-up routine: taken from the
// context's allocator and handed back when the routine ends, once the stream
// has finished with it (the context's arena keeps everything else until
// rt_destroy).
struct Scratch {
  rt_ctx* c;
  std::vector<void*> ptrs;
  explicit Scratch(rt_ctx* ctx) : c(ctx) {}
  template <typename T>
  T* get_n(size_t n) {
    void* p = c->alloc.get(n * sizeof(T) + 16, c->ws);
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Scratch() {
    if (ptrs.empty()) return;
    cudaStreamSynchronize(c->ws);
    for (void* p : ptrs) c->alloc.put(p, c->ws);
  }
};

static GemmArgs args(const void* A, const void* B, void* C) {
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.C = C;
  return g;
}

// residual ||I - Y||_F / sqrt(n) from the per-item partials of an EPI_TWO_I product
static void residual_from_items(rt_ctx* c, Sys& s, const TripleInfo& ti, double* out, double* out2) {
  run(
      c, PC_MISC, 0, 0,
      [&] { launch_sum(s.red_items, ti.t.n_items, s.red_part, std::sqrt((double)s.n_true), out, out2, c->ws); }, 2);
}

// ----------------------------------------------------------------------------
// set-up
// ----------------------------------------------------------------------------
static void upload_padded(rt_ctx* c, Sys& s, const Pattern& P, const double* h_val, double* d_val,
                          bool identity_pad) {
  const int B = s.B;
  std::vector<double> buf((size_t)P.nnzb * B * B, 0.0);
  size_t o = 0;
  for (int i = 0; i < s.n_atoms; ++i) {
    for (int q = P.h_rowptr[i]; q < P.h_rowptr[i + 1]; ++q) {
      int j = P.h_col[q];
      int bi = s.bsize[i], bj = s.bsize[j];
      double* blk = buf.data() + (size_t)q * B * B;
      for (int a = 0; a < bi; ++a)
        for (int b = 0; b < bj; ++b) blk[a * B + b] = h_val[o + (size_t)a * bj + b];
      if (identity_pad && i == j)
        for (int a = bi; a < B; ++a) blk[a * B + a] = 1.0;
      o += (size_t)bi * bj;
    }
  }
  RT_CUDA_CHECK(cudaMemcpyAsync(d_val, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, c->ws));
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
}

static int pad_size(int bmax) {
  if (bmax <= 1) return 1;
  if (bmax <= 4) return 4;
  if (bmax <= 13) return 13;
  return -1;
}

static void setup_system(rt_ctx* c, Sys& s, const rt_system& in) {
  const rt_params& p = c->p;
  RT_REQUIRE(in.n_atoms > 0, RT_EINVAL, "n_atoms must be positive");
  RT_REQUIRE(in.pos && in.bsize && in.s_rowptr && in.s_col && in.s_val && in.h_rowptr && in.h_col && in.h_val,
             RT_EINVAL, "NULL input array");
  RT_REQUIRE(in.d_val[0] && in.d_val[1] && in.d_val[2], RT_EINVAL, "NULL dipole array");
  s.n_atoms = in.n_atoms;
  s.bsize.assign(in.bsize, in.bsize + in.n_atoms);
  int bmax = 0;
  s.n_true = 0;
  for (int b : s.bsize) {
    RT_REQUIRE(b >= 1 && b <= 13, RT_EINVAL, "bsize must be in 1..13");
    bmax = std::max(bmax, b);
    s.n_true += b;
  }
  s.B = pad_size(bmax);
  s.periodic = in.cell != nullptr;
  if (s.periodic) {
    for (int d = 0; d < 3; ++d) {
      s.cell[d] = in.cell[d];
      RT_REQUIRE(s.cell[d] > 0, RT_EINVAL, "cell lengths must be positive");
    }
  }
  s.r_S = in.r_S;
  s.r_H = in.r_H;
  RT_REQUIRE(s.r_S > 0 && s.r_H > 0, RT_EINVAL, "r_S and r_H must be positive");
  s.h_pos.assign(in.pos, in.pos + 3 * (size_t)in.n_atoms);
  for (int i = 0; i < s.n_atoms; ++i)
    for (int d = 0; d < 3; ++d) {
      double x = s.h_pos[3 * i + d];
      RT_REQUIRE(std::isfinite(x), RT_EINVAL, "non-finite position");
      if (s.periodic) RT_REQUIRE(x >= 0.0 && x < s.cell[d], RT_EINVAL, "positions must be wrapped into [0, cell)");
    }
  s.d_pos = c->arena.get_n<double>(3 * (size_t)s.n_atoms);
  s.d_bsize = c->arena.get_n<int32_t>(s.n_atoms);
  RT_CUDA_CHECK(cudaMemcpyAsync(s.d_pos, s.h_pos.data(), sizeof(double) * 3 * s.n_atoms, cudaMemcpyHostToDevice, c->ws));
  RT_CUDA_CHECK(cudaMemcpyAsync(s.d_bsize, s.bsize.data(), sizeof(int32_t) * s.n_atoms, cudaMemcpyHostToDevice, c->ws));

  // given patterns
  s.pS_given = std::make_unique<Pattern>();
  s.pH_given = std::make_unique<Pattern>();
  upload_pattern(*s.pS_given, s.n_atoms, in.s_rowptr, in.s_col, s.r_S, c->arena, c->ws);
  upload_pattern(*s.pH_given, s.n_atoms, in.h_rowptr, in.h_col, s.r_H, c->arena, c->ws);
  s.pS = s.pS_given.get();
  s.pH = s.pH_given.get();
  // built patterns
  s.pSinv = pattern_for(c, s, p.r_Sinv);
  s.pT = pattern_for(c, s, p.r_T);
  s.pU = pattern_for(c, s, p.r_U);
  s.pK = pattern_for(c, s, p.r_K);
  s.pM = pattern_for(c, s, p.r_M);
  s.pA = pattern_for(c, s, std::max(s.r_S, s.r_H));

  // values
  s.S = c->arena.get_n<double>(nvals(s, s.pS));
  s.H0 = c->arena.get_n<double>(nvals(s, s.pH));
  s.Hm = c->arena.get_n<double>(nvals(s, s.pH));
  upload_padded(c, s, *s.pS, in.s_val, s.S, true);
  upload_padded(c, s, *s.pH, in.h_val, s.H0, false);
  for (int d = 0; d < 3; ++d) {
    s.D[d] = c->arena.get_n<double>(nvals(s, s.pH));
    upload_padded(c, s, *s.pH, in.d_val[d], s.D[d], false);
  }
  // matrices of the step
  s.Sinv = c->arena.get_n<double>(nvals(s, s.pSinv));
  s.Zs = c->arena.get_n<double>(nvals(s, s.pSinv));
  s.Xs2 = c->arena.get_n<double>(nvals(s, s.pSinv));
  s.T = c->arena.get_n<double>(nvals(s, s.pT));
  s.P0 = c->arena.get_n<double>(nvals(s, s.pU));
  s.P1 = c->arena.get_n<double>(nvals(s, s.pU));
  s.U = c->arena.get_n<double2>(nvals(s, s.pU));
  s.M = c->arena.get_n<double2>(nvals(s, s.pM));
  for (int k = 0; k < p.n_kick; ++k) {
    double2* Kk = c->arena.get_n<double2>(nvals(s, s.pK));
    RT_CUDA_CHECK(cudaMemsetAsync(Kk, 0, sizeof(double2) * nvals(s, s.pK), c->ws));
    s.K.push_back(Kk);
  }
  s.red_part = c->arena.get_n<double>(1024 * 8);
  s.scal = c->arena.get_n<double>(16);
  s.rows_tmp = c->arena.get_n<double>((size_t)s.n_atoms * s.B);

  // maps
  if (s.pU != s.pT) s.u_to_t = block_map(c, s.pU, s.pT, false);
  s.k_to_sT = block_map(c, s.pK, s.pS, true);
  s.k_to_hT = block_map(c, s.pK, s.pH, true);
  s.u_to_sinv = block_map(c, s.pU, s.pSinv, false);
  s.k_to_sinv = block_map(c, s.pK, s.pSinv, false);
  if (s.pK != s.pM) {
    s.k_to_m = block_map(c, s.pK, s.pM, false);
    s.m_to_k = block_map(c, s.pM, s.pK, false);
  }

  // triple lists of the step
  triples_for(c, s, s.pS, false, s.pSinv, false, s.pSinv, false);   // S X
  triples_for(c, s, s.pSinv, false, s.pSinv, false, s.pSinv, false);  // X Z
  triples_for(c, s, s.pSinv, false, s.pH, false, s.pT, false);      // T = S^-1 H
  triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);         // M = U K
  triples_for(c, s, s.pM, false, s.pU, true, s.pK, true);           // K' = M U^dagger
  if (p.prop != RT_PROP_CN) {
    triples_for(c, s, s.pT, false, s.pT, false, s.pU, false);  // T^2 (M4: T1 T2, T2 T1)
    triples_for(c, s, s.pT, false, s.pU, false, s.pU, false);  // T^n
  }
  if (p.prop == RT_PROP_ETRS || p.prop == RT_PROP_M4) {
    // ETRS: the two half-step exponentials; M4: Om and two power buffers
    s.X = c->arena.get_n<double2>(nvals(s, s.pU));
    s.Xn = c->arena.get_n<double2>(nvals(s, s.pU));
    triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);  // complex products on P_U
    if (p.prop == RT_PROP_M4) {
      s.Zc = c->arena.get_n<double2>(nvals(s, s.pU));
      s.T2 = c->arena.get_n<double>(nvals(s, s.pT));
    }
  }
  if (p.prop == RT_PROP_CN) {
    s.a_to_s = block_map(c, s.pA, s.pS, false);
    s.a_to_h = block_map(c, s.pA, s.pH, false);
    s.Acn = c->arena.get_n<double2>(nvals(s, s.pA));
    s.Bcn = c->arena.get_n<double2>(nvals(s, s.pA));
    s.X = c->arena.get_n<double2>(nvals(s, s.pU));
    s.Xn = c->arena.get_n<double2>(nvals(s, s.pU));
    s.Zc = c->arena.get_n<double2>(nvals(s, s.pU));
    triples_for(c, s, s.pA, false, s.pU, false, s.pU, false);  // A X
    triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);  // X Z
    triples_for(c, s, s.pU, false, s.pA, false, s.pU, false);  // X B
  }
  if (p.precision == RT_FP32 && s.B == 13 && p.tensor_cores) {
    // row tiles of the sandwich's two complex products for the tensor-core kernel
    TripleInfo& tM = triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);
    build_tiles(tM.tiles, tM.t, *s.pM, c->arena, c->ws);
    TripleInfo& tK = triples_for(c, s, s.pM, false, s.pU, true, s.pK, true);
    build_tiles(tK.tiles, tK.t, *s.pK, c->arena, c->ws);
  }
  if (p.precision == RT_FP32) {
    RT_REQUIRE(p.r_M >= p.r_K, RT_EINVAL, "the FP32 delta-form sandwich needs r_M >= r_K");
    s.dUf = c->arena.get_n<float2>(nvals32(s, s.pU));
    if (s.B == 13) s.dUH = c->arena.get_n<float2>(nvals32(s, s.pU));
    s.Kf = c->arena.get_n<float2>(nvals32(s, s.pK));
    s.Mf = c->arena.get_n<float2>(nvals32(s, s.pM));
    s.Wf = c->arena.get_n<float2>(nvals32(s, s.pM));
    // the padding columns of 13-function FP32 blocks are never written: zero them once
    RT_CUDA_CHECK(cudaMemsetAsync(s.dUf, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
    if (s.dUH) RT_CUDA_CHECK(cudaMemsetAsync(s.dUH, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
    RT_CUDA_CHECK(cudaMemsetAsync(s.Kf, 0, sizeof(float2) * nvals32(s, s.pK), c->ws));
    RT_CUDA_CHECK(cudaMemsetAsync(s.Mf, 0, sizeof(float2) * nvals32(s, s.pM), c->ws));
    RT_CUDA_CHECK(cudaMemsetAsync(s.Wf, 0, sizeof(float2) * nvals32(s, s.pM), c->ws));
    if (p.prop == RT_PROP_CN && p.hot_step_iters > p.hot_fp64_iters) {
      s.Acn32 = c->arena.get_n<float2>(nvals32(s, s.pA));
      s.X32 = c->arena.get_n<float2>(nvals32(s, s.pU));
      s.Y32 = c->arena.get_n<float2>(nvals32(s, s.pU));
      s.Xn32 = c->arena.get_n<float2>(nvals32(s, s.pU));
      for (float2* b : {s.X32, s.Y32, s.Xn32})  // padding columns stay zero
        RT_CUDA_CHECK(cudaMemsetAsync(b, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Acn32, 0, sizeof(float2) * nvals32(s, s.pA), c->ws));
    }
    if (p.prop == RT_PROP_ETRS || p.prop == RT_PROP_M4) {
      s.dUa = c->arena.get_n<float2>(nvals32(s, s.pU));
      s.dUb = c->arena.get_n<float2>(nvals32(s, s.pU));
      RT_CUDA_CHECK(cudaMemsetAsync(s.dUa, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.dUb, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
    }
    if (p.prop == RT_PROP_M4) {
      s.Omf = c->arena.get_n<float2>(nvals32(s, s.pU));
      s.Tf2 = c->arena.get_n<float>(nvals32(s, s.pT));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Omf, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Tf2, 0, sizeof(float) * nvals32(s, s.pT), c->ws));
    }
    if (p.prop != RT_PROP_CN) {
      s.Tf = c->arena.get_n<float>(nvals32(s, s.pT));
      s.Pf0 = c->arena.get_n<float>(nvals32(s, s.pU));
      s.Pf1 = c->arena.get_n<float>(nvals32(s, s.pU));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Tf, 0, sizeof(float) * nvals32(s, s.pT), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Pf0, 0, sizeof(float) * nvals32(s, s.pU), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Pf1, 0, sizeof(float) * nvals32(s, s.pU), c->ws));
      s.T0 = c->arena.get_n<double>(nvals(s, s.pT));
      s.TD = c->arena.get_n<double>(nvals(s, s.pT));
    }
  }
  if (p.field_poly) {
    RT_REQUIRE(p.prop == RT_PROP_EM, RT_EINVAL, "the field polynomial is defined for the EM propagator");
    if (!s.T0) s.T0 = c->arena.get_n<double>(nvals(s, s.pT));
    s.TDn = c->arena.get_n<double>(nvals(s, s.pT));
    for (int m = 0; m < p.taylor_terms; ++m) s.V.push_back(c->arena.get_n<double2>(nvals(s, s.pU)));
  }
  if (p.incremental) {
    // reference split K = K_ref + dK (block sizes 4 and 13: the FP32 kernels that take R)
    RT_REQUIRE(s.B == 13 || s.B == 4, RT_EINVAL, "the reference split needs block size 4 or 13");
    s.Kref = c->arena.get_n<double2>(nvals(s, s.pK));
    s.Rm = c->arena.get_n<double2>(nvals(s, s.pK));
    s.tref = c->arena.get_n<double>(8);
    for (int k = 0; k < p.n_kick; ++k) s.dK.push_back(c->arena.get_n<double2>(nvals(s, s.pK)));
    s.dk_fresh.assign(p.n_kick, 0);
    if (p.full_step) {
      // coefficients B_0..B_2deg of R(E), formed with the reference (first step)
      const int deg = p.taylor_terms - 1;
      RT_REQUIRE(2 * deg < RT_MAX_POLY, RT_EINVAL, "taylor_terms too large for the reference split");
      for (int q = 0; q <= 2 * deg; ++q) s.Bp.push_back(c->arena.get_n<double2>(nvals(s, s.pK)));
      s.d_bp = c->arena.get_n<double2*>(s.Bp.size());
      RT_CUDA_CHECK(
          cudaMemcpyAsync(s.d_bp, s.Bp.data(), sizeof(double2*) * s.Bp.size(), cudaMemcpyHostToDevice, c->ws));
    }
    s.Kfk.push_back(s.Kf);
    s.Mfk.push_back(s.Mf);
    s.Wfk.push_back(s.Wf);
    for (int k = 1; k < p.n_kick; ++k) {
      s.Kfk.push_back(c->arena.get_n<float2>(nvals32(s, s.pK)));
      s.Mfk.push_back(c->arena.get_n<float2>(nvals32(s, s.pM)));
      s.Wfk.push_back(c->arena.get_n<float2>(nvals32(s, s.pM)));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Kfk.back(), 0, sizeof(float2) * nvals32(s, s.pK), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Mfk.back(), 0, sizeof(float2) * nvals32(s, s.pM), c->ws));
      RT_CUDA_CHECK(cudaMemsetAsync(s.Wfk.back(), 0, sizeof(float2) * nvals32(s, s.pM), c->ws));
    }
    s.dUr = c->arena.get_n<float2>(nvals32(s, s.pU));
    RT_CUDA_CHECK(cudaMemsetAsync(s.dUr, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
    if (s.B == 13) {  // the 13-function kernels read a pre-transposed dagger
      s.dUHr = c->arena.get_n<float2>(nvals32(s, s.pU));
      RT_CUDA_CHECK(cudaMemsetAsync(s.dUHr, 0, sizeof(float2) * nvals32(s, s.pU), c->ws));
      s.planar = p.packed_fma != 0 && !p.tensor_cores;
    }
  }
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
}

static void build_field_poly(rt_ctx* c, Sys& s);

// ----------------------------------------------------------------------------
// Hotelling inverse of S (Sec. V.A), cut to r_Sinv
// ----------------------------------------------------------------------------
static rt_status hotelling_sinv(rt_ctx* c, Sys& s) {
  const rt_params& p = c->p;
  Pattern* P = s.pSinv;
  TripleInfo& tSX = triples_for(c, s, s.pS, false, P, false, P, false);
  TripleInfo& tXZ = triples_for(c, s, P, false, P, false, P, false);
  launch_inf_norm(s.S, s.pS->rowptr, s.pS->col, s.d_bsize, s.B, s.n_atoms, s.rows_tmp, s.scal, c->ws);
  double nrm = 0.0;
  RT_CUDA_CHECK(cudaMemcpyAsync(&nrm, s.scal, sizeof(double), cudaMemcpyDeviceToHost, c->ws));
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
  RT_REQUIRE(nrm > 0 && std::isfinite(nrm), RT_ENUMERIC, "||S||_inf is not a positive finite number");
  launch_identity(s.Sinv, false, P->nnzb, P->rowidx, P->col, s.B, 1.0 / nrm, c->ws);
  double prev = -1.0, res = 0.0;
  int it = 0;
  rt_status status = RT_OK;
  s.sinv_status = "maxit";
  for (;;) {
    // Z = 2I - S X, residual ||I - S X||
    GemmArgs g = args(s.S, s.Sinv, s.Zs);
    g.red = s.red_items;
    gemm(c, s, PC_MISC, tSX, false, false, false, false, EPI_TWO_I, g, P);
    residual_from_items(c, s, tSX, s.scal, nullptr);
    RT_CUDA_CHECK(cudaMemcpyAsync(&res, s.scal, sizeof(double), cudaMemcpyDeviceToHost, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    if (!std::isfinite(res) || res > 1.0) {
      s.sinv_status = "diverged";
      status = RT_ENOTCONV;
      break;
    }
    if (res < p.hot_tol) {
      s.sinv_status = "converged";
      break;
    }
    if (prev >= 0.0 && res > 0.9 * prev) {
      s.sinv_status = "stagnated";
      break;
    }
    if (it >= p.hot_maxit) {
      status = RT_ENOTCONV;
      break;
    }
    // X <- X Z
    gemm(c, s, PC_MISC, tXZ, false, false, false, false, EPI_STORE, args(s.Sinv, s.Zs, s.Xs2), P);
    std::swap(s.Sinv, s.Xs2);
    prev = res;
    ++it;
  }
  s.sinv_iters = it;
  s.sinv_resid = res;
  s.sinv_ready = true;
  if (s.X) launch_restrict(s.Sinv, (double*)s.X, s.u_to_sinv, s.pU->nnzb, s.B, 1, c->ws);
  if (c->p.precision == RT_FP32 && c->p.prop != RT_PROP_CN) {
    // T0 = cut(S^-1 H0) and T_D = cut(S^-1 D_dir): T(t) = T0 - E(t) T_D exactly
    TripleInfo& tT = triples_for(c, s, P, false, s.pH, false, s.pT, false);
    gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.H0, s.T0), s.pT);
    gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.D[c->field.dir], s.TD), s.pT);
  }
  if (c->p.field_poly) build_field_poly(c, s);
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
  c->graph_dirty = true;
  return status;
}

// ----------------------------------------------------------------------------
// propagator
// ----------------------------------------------------------------------------
static void taylor_coef(int n, double dt, double* mag, int* imag) {
  // (-i dt)^n / n!: (-i)^n = 1, -i, -1, i for n mod 4 = 0..3
  double v = 1.0;
  for (int k = 1; k <= n; ++k) v *= dt / k;
  switch (n % 4) {
    case 0: *mag = v; *imag = 0; break;
    case 1: *mag = -v; *imag = 1; break;
    case 2: *mag = -v; *imag = 0; break;
    default: *mag = v; *imag = 1; break;
  }
}

// U = sum_{n<terms} c_n T^n with T real on P_T, powers cut to P_U.  FP64 U
// (into Uout, default s.U) or the FP32 difference dU = U - I (into dUout;
// by default s.dUf, with (U - I)^dagger into s.dUH where that exists).
static void taylor_series(rt_ctx* c, Sys& s, const double* T, double dt, int terms, bool fp32_delta,
                          double2* Uout = nullptr, float2* dUout = nullptr) {
  if (!Uout) Uout = s.U;
  float2* dUH = dUout ? nullptr : s.dUH;
  if (!dUout) dUout = s.dUf;
  TripleInfo& t2 = triples_for(c, s, s.pT, false, s.pT, false, s.pU, false);
  TripleInfo& tn = triples_for(c, s, s.pT, false, s.pU, false, s.pU, false);
  double c1 = 0.0;
  int c1i = 0;
  taylor_coef(1, dt, &c1, &c1i);
  if (!fp32_delta) {
    run(c, PC_MISC, 0, 0, [&] {
      launch_taylor_init(Uout, false, s.pU->nnzb, s.pU->rowidx, s.pU->col, T, false, s.u_to_t, s.B,
                         terms > 1 ? c1 : 0.0, c1i, 1, c->ws);
    });
    const double* prev = T;
    double* bufs[2] = {s.P0, s.P1};
    for (int n = 2; n < terms; ++n) {
      double cn;
      int ci;
      taylor_coef(n, dt, &cn, &ci);
      GemmArgs g = args(T, prev, bufs[n % 2]);
      g.U = Uout;
      g.coef = cn;
      g.coef_imag = ci;
      gemm(c, s, PC_TAYLOR, n == 2 ? t2 : tn, false, false, false, false, EPI_STORE_ACC, g, s.pU);
      prev = bufs[n % 2];
    }
  } else {
    run(
        c, PC_MISC, 0, 0,
        [&] {
          launch_d2f_pad(T, s.Tf, s.pT->nnzb, s.B, false, c->ws);
          launch_taylor_init(dUout, true, s.pU->nnzb, s.pU->rowidx, s.pU->col, T, false, s.u_to_t, s.B,
                             terms > 1 ? c1 : 0.0, c1i, 0, c->ws);
        },
        2);
    const float* prev = s.Tf;
    float* bufs[2] = {s.Pf0, s.Pf1};
    for (int n = 2; n < terms; ++n) {
      double cn;
      int ci;
      taylor_coef(n, dt, &cn, &ci);
      // the last power is needed only inside U: no store of C; its epilogue
      // also writes (U - I)^dagger per block for the sandwich (13-function
      // kernels; the generic kernel takes the transpose while staging)
      const bool last = n == terms - 1;
      GemmArgs g = args(s.Tf, prev, last ? nullptr : bufs[n % 2]);
      g.U = dUout;
      g.coef = cn;
      g.coef_imag = ci;
      if (last && dUH) g.base = dUH;
      gemm(c, s, PC_TAYLOR, n == 2 ? t2 : tn, true, false, false, false, EPI_STORE_ACC, g, s.pU);
      prev = bufs[n % 2];
    }
    if (dUH && terms < 3) run(c, PC_MISC, 0, 0, [&] { launch_dagger32(dUout, dUH, s.pU->nnzb, s.B, c->ws); });
  }
}

// field samples of the device step state (k_begin_step)
enum { E_MID = 0, E_T = 1, E_TDT = 2, E_T1 = 3, E_T2 = 4 };

// H = H0 - E(t_which) D_j into s.Hm
static void field_hamiltonian(rt_ctx* c, Sys& s, int which) {
  const int dir = c->field.dir;
  run(c, PC_FIELD, 0, 24.0 * nvals(s, s.pH),
      [&] { launch_field_axpy(s.H0, s.D[dir], c->dstate, which, 1.0, s.Hm, (int64_t)nvals(s, s.pH), c->ws); });
}

// T = cut_{r_T}(S^-1 H(t_which)) into Tout
static void field_T(rt_ctx* c, Sys& s, int which, double* Tout) {
  field_hamiltonian(c, s, which);
  TripleInfo& tT = triples_for(c, s, s.pSinv, false, s.pH, false, s.pT, false);
  gemm(c, s, PC_T, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.Hm, Tout), s.pT);
}

// ETRS (Sec. II.A): U = cut(exp(-i dt/2 T(t+dt)) exp(-i dt/2 T(t))), each
// exponential by the truncated Taylor series.  Mixed mode: with the FP32
// differences dU_a = exp(-i dt/2 T(t)) - I and dU_b = exp(-i dt/2 T(t+dt)) - I
// (both on P_U, which holds the identity blocks), the cut is linear, so
//   U - I = dU_a + dU_b + cut(dU_b dU_a)
// exactly; the fields enter through T(t) = T0 - E(t) T_D.
static void build_etrs(rt_ctx* c, Sys& s, bool fp32) {
  const rt_params& p = c->p;
  if (fp32) {
    const int64_t nT = (int64_t)nvals(s, s.pT);
    run(c, PC_FIELD, 0, 16.0 * nT, [&] { launch_field_axpy(s.T0, s.TD, c->dstate, E_T, 1.0, s.T, nT, c->ws); });
    taylor_series(c, s, s.T, 0.5 * p.dt, p.taylor_terms, true, nullptr, s.dUa);
    run(c, PC_FIELD, 0, 16.0 * nT, [&] { launch_field_axpy(s.T0, s.TD, c->dstate, E_TDT, 1.0, s.T, nT, c->ws); });
    taylor_series(c, s, s.T, 0.5 * p.dt, p.taylor_terms, true, nullptr, s.dUb);
    const int64_t nU = (int64_t)nvals32(s, s.pU);
    run(c, PC_MISC, 0, 0, [&] { launch_axpy32(s.dUf, s.dUa, s.dUb, 1.0f, nU, c->ws); });
    TripleInfo& tUU = triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);
    gemm(c, s, PC_TAYLOR, tUU, true, true, false, false, EPI_ADD, args(s.dUb, s.dUa, s.dUf), s.pU);
    if (s.dUH) run(c, PC_MISC, 0, 0, [&] { launch_dagger32(s.dUf, s.dUH, s.pU->nnzb, s.B, c->ws); });
    s.duf_current = true;
    return;
  }
  field_T(c, s, E_T, s.T);
  taylor_series(c, s, s.T, 0.5 * p.dt, p.taylor_terms, false, s.X);
  field_T(c, s, E_TDT, s.T);
  taylor_series(c, s, s.T, 0.5 * p.dt, p.taylor_terms, false, s.Xn);
  TripleInfo& tUU = triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);
  gemm(c, s, PC_TAYLOR, tUU, false, true, false, false, EPI_STORE, args(s.Xn, s.X, s.U), s.pU);
}

// fourth-order Magnus (Sec. II.A): T1, T2 at t + (1/2 -+ sqrt(3)/6) dt,
// Om = -i dt/2 (T1 + T2) - sqrt(3) dt^2/12 [T2, T1] on P_U,
// U = sum_{n<terms} Om^n / n! with Om^n = cut(Om Om^{n-1})
static void build_m4(rt_ctx* c, Sys& s, bool fp32) {
  const rt_params& p = c->p;
  if (fp32) {
    // mixed mode: T1, T2 = T0 - E(t1,2) T_D; the commutator products and the
    // powers of Om as FP32 block products; dU = exp(Om) - I accumulated in
    // FP32 (the identity is never added, as in the other delta forms)
    const int64_t nT = (int64_t)nvals(s, s.pT);
    run(
        c, PC_FIELD, 0, 32.0 * nT,
        [&] {
          launch_field_axpy(s.T0, s.TD, c->dstate, E_T1, 1.0, s.T, nT, c->ws);
          launch_field_axpy(s.T0, s.TD, c->dstate, E_T2, 1.0, s.T2, nT, c->ws);
        },
        2);
    run(
        c, PC_MISC, 0, 0,
        [&] {
          launch_d2f_pad(s.T, s.Tf, s.pT->nnzb, s.B, false, c->ws);
          launch_d2f_pad(s.T2, s.Tf2, s.pT->nnzb, s.B, false, c->ws);
        },
        2);
    TripleInfo& tTT = triples_for(c, s, s.pT, false, s.pT, false, s.pU, false);
    gemm(c, s, PC_TAYLOR, tTT, true, false, false, false, EPI_STORE, args(s.Tf2, s.Tf, s.Pf0), s.pU);  // T2 T1
    gemm(c, s, PC_TAYLOR, tTT, true, false, false, false, EPI_STORE, args(s.Tf, s.Tf2, s.Pf1), s.pU);  // T1 T2
    run(c, PC_MISC, 0, 0, [&] {
      launch_m4_omega32(s.T, s.T2, s.u_to_t, s.Pf0, s.Pf1, p.dt, s.Omf, s.dUf, p.taylor_terms > 1, s.pU->nnzb, s.B,
                        c->ws);
    });
    TripleInfo& tUU = triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);
    const int64_t nU = (int64_t)nvals32(s, s.pU);
    const float2* prev = s.Omf;
    float2* bufs[2] = {s.dUa, s.dUb};
    double inv_fact = 1.0;
    for (int n = 2; n < p.taylor_terms; ++n) {
      inv_fact /= n;
      float2* out = bufs[n % 2];
      gemm(c, s, PC_TAYLOR, tUU, true, true, false, false, EPI_STORE, args(s.Omf, prev, out), s.pU);
      run(c, PC_MISC, 0, 0, [&] { launch_axpy32(s.dUf, s.dUf, out, (float)inv_fact, nU, c->ws); });
      prev = out;
    }
    if (s.dUH) run(c, PC_MISC, 0, 0, [&] { launch_dagger32(s.dUf, s.dUH, s.pU->nnzb, s.B, c->ws); });
    s.duf_current = true;
    return;
  }
  field_T(c, s, E_T1, s.T);
  field_T(c, s, E_T2, s.T2);
  TripleInfo& tTT = triples_for(c, s, s.pT, false, s.pT, false, s.pU, false);
  gemm(c, s, PC_TAYLOR, tTT, false, false, false, false, EPI_STORE, args(s.T2, s.T, s.P0), s.pU);  // T2 T1
  gemm(c, s, PC_TAYLOR, tTT, false, false, false, false, EPI_STORE, args(s.T, s.T2, s.P1), s.pU);  // T1 T2
  const int64_t nu = (int64_t)nvals(s, s.pU);
  run(
      c, PC_MISC, 0, 0,
      [&] {
        launch_m4_omega(s.T, s.T2, s.u_to_t, s.P0, s.P1, p.dt, s.Zc, s.pU->nnzb, s.B, c->ws);
        launch_identity((double*)s.U, true, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, 1.0, c->ws);
        if (p.taylor_terms > 1) launch_zaxpy(s.U, s.U, s.Zc, 1.0, nu, c->ws);
      },
      p.taylor_terms > 1 ? 3 : 2);
  TripleInfo& tUU = triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);
  const double2* prev = s.Zc;
  double2* bufs[2] = {s.X, s.Xn};
  double inv_fact = 1.0;
  for (int n = 2; n < p.taylor_terms; ++n) {
    inv_fact /= n;
    double2* out = bufs[n % 2];
    gemm(c, s, PC_TAYLOR, tUU, false, true, false, false, EPI_STORE, args(s.Zc, prev, out), s.pU);
    run(c, PC_MISC, 0, 0, [&] { launch_zaxpy(s.U, s.U, out, inv_fact, nu, c->ws); });
    prev = out;
  }
}

// Coefficients of the EM propagator as a polynomial in the field value E
// (H = H0 - E D, eq. EM with every product cut as in the literal series):
// T(E) = Q_{1,0} + E Q_{1,1} with Q_{1,0} = cut(S^-1 H0), Q_{1,1} = -cut(S^-1 D);
// T^n(E) = cut(T(E) T^{n-1}(E)) = sum_m E^m Q_{n,m} with
// Q_{n,m} = cut(Q_{1,0} Q_{n-1,m}) + cut(Q_{1,1} Q_{n-1,m-1}) (the cut is linear);
// U(E) = I + sum_n c_n T^n(E) = sum_m E^m V_m, V_m = sum_n c_n Q_{n,m} (+ I in V_0).
static void build_field_poly(rt_ctx* c, Sys& s) {
  const rt_params& p = c->p;
  s.r_ready = false;  // the reference split's B_p follow the V_m
  const int deg = p.taylor_terms - 1;
  Pattern* PT = s.pT;
  Pattern* PU = s.pU;
  const size_t nT = nvals(s, PT), nU = nvals(s, PU);
  TripleInfo& tT = triples_for(c, s, s.pSinv, false, s.pH, false, PT, false);
  gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.H0, s.T0), PT);
  gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.D[c->field.dir], s.TDn), PT);
  launch_scale(s.TDn, -1.0, (int64_t)nT, c->ws);
  launch_identity(reinterpret_cast<double*>(s.V[0]), true, PU->nnzb, PU->rowidx, PU->col, s.B, 1.0, c->ws);
  for (int m = 1; m <= deg; ++m) RT_CUDA_CHECK(cudaMemsetAsync(s.V[m], 0, sizeof(double2) * nU, c->ws));
  if (deg >= 1) {
    double c1 = 0.0;
    int i1 = 0;
    taylor_coef(1, p.dt, &c1, &i1);
    launch_acc_real(s.V[0], s.T0, s.u_to_t, PU->nnzb, s.B, c1, i1, c->ws);
    launch_acc_real(s.V[1], s.TDn, s.u_to_t, PU->nnzb, s.B, c1, i1, c->ws);
  }
  Scratch tmp(c);  // coefficient matrices of two consecutive powers while the V_m are formed
  std::vector<double*> Qa, Qb;
  if (deg >= 2)
    for (int m = 0; m <= deg; ++m) {
      Qa.push_back(tmp.get_n<double>(nU));
      Qb.push_back(tmp.get_n<double>(nU));
    }
  TripleInfo& t2 = triples_for(c, s, PT, false, PT, false, PU, false);
  TripleInfo& tn = triples_for(c, s, PT, false, PU, false, PU, false);
  std::vector<const double*> prev = {s.T0, s.TDn};
  for (int n = 2; n <= deg; ++n) {
    TripleInfo& tl = n == 2 ? t2 : tn;
    double cn = 0.0;
    int ci = 0;
    taylor_coef(n, p.dt, &cn, &ci);
    std::vector<double*>& out = (n % 2 == 0) ? Qa : Qb;
    for (int m = 0; m <= n; ++m) {
      bool first = true;
      if (m <= n - 1) {
        gemm(c, s, PC_MISC, tl, false, false, false, false, EPI_STORE, args(s.T0, prev[m], out[m]), PU);
        first = false;
      }
      if (m >= 1)
        gemm(c, s, PC_MISC, tl, false, false, false, false, first ? EPI_STORE : EPI_ADD,
             args(s.TDn, prev[m - 1], out[m]), PU);
      launch_acc_real(s.V[m], out[m], nullptr, PU->nnzb, s.B, cn, ci, c->ws);
    }
    prev.assign(out.begin(), out.begin() + n + 1);
  }
  if (p.incremental && p.precision == RT_FP32) {
    // FP32 copies of V_1..V_deg for the per-step pass of the reference split
    if (s.V32.empty()) {
      s.V32.push_back(nullptr);
      for (int m = 1; m <= deg; ++m) s.V32.push_back(c->arena.get_n<float2>(nU));
    }
    for (int m = 1; m <= deg; ++m) launch_z2c(s.V[m], s.V32[m], (int64_t)nU, c->ws);
  }
}

static void build_propagator(rt_ctx* c, Sys& s, bool fp32) {
  const rt_params& p = c->p;
  if (p.prop == RT_PROP_EM && p.field_poly) {
    PolyTerms V;
    memset(&V, 0, sizeof(V));
    const int deg = p.taylor_terms - 1;
    for (int m = 0; m <= deg; ++m) V.v[m] = s.V[m];
    const double nU = (double)nvals(s, s.pU);
    run(c, PC_POLY, 0, 16.0 * nU * (deg + 2), [&] {  // read V_0..V_deg, write U (or dU and dU^dagger)
      launch_field_poly(V, deg, c->dstate, E_MID, fp32 ? nullptr : s.U, fp32 ? s.dUf : nullptr,
                        fp32 ? s.dUH : nullptr, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws);
    });
    s.duf_current = fp32;
    return;
  }
  if (p.prop == RT_PROP_EM) {
    if (fp32) {
      // T(t+dt/2) = T0 - E T_D (linearity of the cut product in E)
      run(c, PC_FIELD, 0, 16.0 * nvals(s, s.pT),
          [&] { launch_field_axpy(s.T0, s.TD, c->dstate, E_MID, 1.0, s.T, (int64_t)nvals(s, s.pT), c->ws); });
      taylor_series(c, s, s.T, p.dt, p.taylor_terms, true);
      s.duf_current = true;
    } else {
      field_T(c, s, E_MID, s.T);
      taylor_series(c, s, s.T, p.dt, p.taylor_terms, false);
    }
    return;
  }
  if (p.prop == RT_PROP_ETRS || p.prop == RT_PROP_M4) {
    if (p.prop == RT_PROP_ETRS) build_etrs(c, s, fp32);
    else build_m4(c, s, fp32);
    if (fp32) return;
  } else {
    field_hamiltonian(c, s, E_MID);
    run(c, PC_FIELD, 0, 48.0 * nvals(s, s.pA), [&] {
      launch_cn_operands(s.S, s.a_to_s, s.Hm, s.a_to_h, 0.5 * p.dt, s.Acn, s.Bcn, s.pA->nnzb, s.B, c->ws);
    });
    TripleInfo& tAX = triples_for(c, s, s.pA, false, s.pU, false, s.pU, false);
    TripleInfo& tXZ = triples_for(c, s, s.pU, false, s.pU, false, s.pU, false);
    TripleInfo& tXB = triples_for(c, s, s.pU, false, s.pA, false, s.pU, false);
    // mixed mode: the first iterations as FP32 block products (X rounded to
    // FP32 and back); the last hot_fp64_iters in FP64, with the residual
    const int n32 = (fp32 && s.X32) ? std::max(0, p.hot_step_iters - p.hot_fp64_iters) : 0;
    if (n32 > 0) {
      run(
          c, PC_MISC, 0, 0,
          [&] {
            launch_d2f_pad(reinterpret_cast<const double*>(s.Acn), reinterpret_cast<float*>(s.Acn32), s.pA->nnzb,
                           s.B, true, c->ws);
            launch_d2f_pad(reinterpret_cast<const double*>(s.X), reinterpret_cast<float*>(s.X32), s.pU->nnzb, s.B,
                           true, c->ws);
          },
          2);
      float2* x32[2] = {s.X32, s.Xn32};
      for (int it = 0; it < n32; ++it) {
        float2* xi = x32[it % 2];
        float2* xo = x32[(it + 1) % 2];
        gemm(c, s, PC_CN_HOT, tAX, true, true, false, false, EPI_STORE, args(s.Acn32, xi, s.Y32), s.pU);
        run(c, PC_MISC, 0, 0,
            [&] { launch_two_i_minus32(s.Y32, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws); });
        gemm(c, s, PC_CN_HOT, tXZ, true, true, false, false, EPI_STORE, args(xi, s.Y32, xo), s.pU);
      }
      run(c, PC_MISC, 0, 0, [&] { launch_f2d_unpad(x32[n32 % 2], s.X, s.pU->nnzb, s.B, c->ws); });
    }
    // X alternates between two fixed buffers and ends in s.X, so that a
    // captured step graph can be replayed (no host-side pointer swaps)
    const int n64 = p.hot_step_iters - n32;
    double2* xb[2] = {s.X, s.Xn};
    for (int it = 0; it < n64; ++it) {
      double2* xi = xb[it % 2];
      double2* xo = xb[(it + 1) % 2];
      GemmArgs g = args(s.Acn, xi, s.Zc);
      g.red = s.red_items;
      gemm(c, s, PC_CN_HOT, tAX, false, true, false, false, EPI_TWO_I, g, s.pU);
      if (it == n64 - 1) residual_from_items(c, s, tAX, s.scal + 1, nullptr);
      gemm(c, s, PC_CN_HOT, tXZ, false, true, false, false, EPI_STORE, args(xi, s.Zc, xo), s.pU);
    }
    if (n64 % 2 == 1)
      run(c, PC_MISC, 0, 0, [&] {
        RT_CUDA_CHECK(cudaMemcpyAsync(s.X, s.Xn, sizeof(double2) * nvals(s, s.pU), cudaMemcpyDeviceToDevice, c->ws));
      });
    if (p.hot_step_iters > 0) run(c, PC_MISC, 0, 0, [&] { launch_set_hot(c->dstate, s.scal + 1, p.hot_step_iters, c->ws); });
    gemm(c, s, PC_CN_U, tXB, false, true, false, false, EPI_STORE, args(s.X, s.Bcn, s.U), s.pU);
  }
  if (fp32) {
    // FP64 U; dU = U - I in FP32 for the delta-form sandwich
    run(c, PC_MISC, 0, 0,
        [&] { launch_u_minus_i_f32(s.U, s.dUf, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws); });
    if (s.dUH) run(c, PC_MISC, 0, 0, [&] { launch_dagger32(s.dUf, s.dUH, s.pU->nnzb, s.B, c->ws); });
  }
}


// ----------------------------------------------------------------------------
// sandwich K <- U K U^dagger and observables
// ----------------------------------------------------------------------------
static void sandwich(rt_ctx* c, Sys& s, int kick, int slot) {
  const bool fp32 = c->p.precision == RT_FP32;
  TripleInfo& tM = triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);
  TripleInfo& tK = triples_for(c, s, s.pM, false, s.pU, true, s.pK, true);
  double2* K = s.K[kick];
  unsigned long long* herm = &c->dstate->herm_bits[slot];
  if (!fp32) {
    gemm(c, s, PC_UK, tM, false, true, false, false, EPI_STORE, args(s.U, K, s.M), s.pM);
    GemmArgs g = args(s.M, s.U, K);
    g.herm_max = herm;
    gemm(c, s, PC_MUDAG, tK, false, true, false, true, EPI_SANDWICH, g, s.pK);
  } else {
    // delta form: M = dU K, W = K + M, K' = K + M + W dU^dagger (K, sums in FP64)
    run(c, PC_MISC, 0, 0, [&] { launch_d2f_pad((const double*)K, (float*)s.Kf, s.pK->nnzb, s.B, true, c->ws); });
    if (s.B == 13) {
      // M = dU K with W = K + M written by the same epilogue
      GemmArgs gm = args(s.dUf, s.Kf, s.Mf);
      gm.base = K;
      gm.U = s.Wf;
      gm.add_map = s.m_to_k;
      gemm(c, s, PC_UK, tM, true, true, false, false, EPI_STORE, gm, s.pM);
    } else {
      gemm(c, s, PC_UK, tM, true, true, false, false, EPI_STORE, args(s.dUf, s.Kf, s.Mf), s.pM);
      run(c, PC_MISC, 0, 0, [&] { launch_delta_w(K, s.m_to_k, s.Mf, s.Wf, s.pM->nnzb, s.B, c->ws); });
    }
    // 13-function blocks read a pre-transposed (U - I)^dagger; the generic
    // kernel transposes while staging
    const bool pre_t = s.dUH != nullptr;
    GemmArgs g = args(s.Wf, pre_t ? s.dUH : s.dUf, K);
    g.herm_max = herm;
    g.base = K;
    g.addend = s.Mf;
    g.add_map = s.k_to_m;
    gemm(c, s, PC_MUDAG, tK, true, true, false, !pre_t, EPI_DELTA_SANDWICH, g, s.pK);
  }
}

static void observe(rt_ctx* c, Sys& s, int kick, int slot) {
  double bytes = 16.0 * nvals(s, s.pK) + 8.0 * 4 * nvals(s, s.pH);
  const bool incr = incremental(c);
  run(
      c, PC_OBS, 0, bytes,
      [&] {
        launch_traces(incr ? s.dK[kick] : s.K[kick], s.pK->nnzb, s.pK->rowidx, s.pK->col, s.d_bsize, s.B, s.S,
                      s.k_to_sT, s.D[0], s.D[1], s.D[2], s.k_to_hT, s.red_part, c->dstate, slot, c->ring,
                      c->p.obs_capacity, c->n_slots, slot, c->ws, incr ? s.tref : nullptr, nullptr);
      },
      2);
}

// K = K_ref + dK for the kicks whose K is stale.  keep = false hands K back
// as the authoritative density (the next step forms dK = K - K_ref again);
// a read (keep = true) leaves dK in place, so the run continues unchanged.
static void materialize(rt_ctx* c, Sys& s, bool keep = false) {
  for (size_t k = 0; k < s.dk_fresh.size(); ++k) {
    if (!s.dk_fresh[k]) continue;
    launch_zaxpy(s.K[k], s.Kref, s.dK[k], 1.0, (int64_t)nvals(s, s.pK), c->ws);
    if (!keep) s.dk_fresh[k] = 0;
  }
}

// FP64 U of the last step where only its FP32 rounding was formed (field
// polynomial in the reference split): U = sum_m E^m V_m at the last E(t + dt/2)
static void refresh_u64(rt_ctx* c, Sys& s) {
  if (!s.u64_stale) return;
  PolyTerms V;
  memset(&V, 0, sizeof(V));
  const int deg = c->p.taylor_terms - 1;
  for (int m = 0; m <= deg; ++m) V.v[m] = s.V[m];
  launch_field_poly(V, deg, c->dstate, 0, s.U, nullptr, nullptr, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws);
  s.u64_stale = false;
}

// The reference of a system: K_ref = K of its first kick slot, its traces
// Tr(K_ref X), and the FP64 part of the step that acts on K_ref:
//  * constant U: R = sym(cut(cut(U K_ref) U^dagger)) - K_ref;
//  * field polynomial (U(E) = sum_m E^m V_m): every cut is linear, so
//    sym(cut(cut(U(E) K_ref) U(E)^dagger)) = sum_p E^p B_p with
//    B_p = sum_{m+m'=p} sym(cut(cut(V_m K_ref) V_m'^dagger)); B_0 takes -K_ref,
//    and each step forms R(E) = sum_p E^p B_p by Horner (k_poly_upper).
// Then dK = K - K_ref for every kick slot whose K changed.
static void prepare_reference(rt_ctx* c, Sys& s) {
  const size_t nv = nvals(s, s.pK);
  if (!s.ref_ready) {
    materialize(c, s);
    RT_CUDA_CHECK(cudaMemcpyAsync(s.Kref, s.K[0], sizeof(double2) * nv, cudaMemcpyDeviceToDevice, c->ws));
    launch_traces(s.Kref, s.pK->nnzb, s.pK->rowidx, s.pK->col, s.d_bsize, s.B, s.S, s.k_to_sT, s.D[0], s.D[1],
                  s.D[2], s.k_to_hT, s.red_part, c->dstate, 0, c->ring, c->p.obs_capacity, c->n_slots, 0, c->ws,
                  nullptr, s.tref);
    s.ref_ready = true;
    s.r_ready = false;
  }
  if (!s.r_ready) {
    TripleInfo& tM = triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);
    TripleInfo& tK = triples_for(c, s, s.pM, false, s.pU, true, s.pK, true);
    if (c->p.full_step) {
      const int deg = c->p.taylor_terms - 1;
      RT_REQUIRE((int)s.V.size() == deg + 1, RT_ESTATE, "the field polynomial is not formed (call rt_inverse)");
      RT_REQUIRE(2 * deg < RT_MAX_POLY, RT_EINVAL, "taylor_terms too large for the reference split");
      Scratch tmp(c);  // cut(V_m K_ref) on P_M while the B_p are formed
      std::vector<double2*> Am;
      for (int m = 0; m <= deg; ++m) Am.push_back(tmp.get_n<double2>(nvals(s, s.pM)));
      if (s.Bp.empty())
        for (int q = 0; q <= 2 * deg; ++q) s.Bp.push_back(c->arena.get_n<double2>(nv));
      for (double2* b : s.Bp) RT_CUDA_CHECK(cudaMemsetAsync(b, 0, sizeof(double2) * nv, c->ws));
      for (int m = 0; m <= deg; ++m)
        gemm(c, s, PC_MISC, tM, false, true, false, false, EPI_STORE, args(s.V[m], s.Kref, Am[m]), s.pM);
      for (int m = 0; m <= deg; ++m)
        for (int m2 = 0; m2 <= deg; ++m2) {
          gemm(c, s, PC_MISC, tK, false, true, false, true, EPI_SANDWICH, args(Am[m], s.V[m2], s.Rm), s.pK);
          launch_zaxpy(s.Bp[m + m2], s.Bp[m + m2], s.Rm, 1.0, (int64_t)nv, c->ws);
        }
      launch_zaxpy(s.Bp[0], s.Bp[0], s.Kref, -1.0, (int64_t)nv, c->ws);
    } else {
      gemm(c, s, PC_MISC, tM, false, true, false, false, EPI_STORE, args(s.U, s.Kref, s.M), s.pM);
      gemm(c, s, PC_MISC, tK, false, true, false, true, EPI_SANDWICH, args(s.M, s.U, s.Rm), s.pK);
      launch_zaxpy(s.Rm, s.Rm, s.Kref, -1.0, (int64_t)nv, c->ws);
    }
    s.r_ready = true;
  }
  for (size_t k = 0; k < s.dk_fresh.size(); ++k) {
    if (s.dk_fresh[k]) continue;
    launch_zaxpy(s.dK[k], s.K[k], s.Kref, -1.0, (int64_t)nv, c->ws);
    launch_d2f_pad((const double*)s.dK[k], (float*)s.Kfk[k], s.pK->nnzb, s.B, true, c->ws);
    s.dk_fresh[k] = 1;
  }
}

// With the field polynomial on the CUDA cores, the K' epilogue evaluates
// R(E) = sum_p E^p B_p itself (the tensor-core kernel reads R from the
// separate Horner pass).
static bool r_fused(const rt_ctx* c, const Sys& s) {
  return incremental(c) && c->p.full_step && s.d_bp != nullptr &&
         !(c->p.precision == RT_FP32 && c->p.tensor_cores && s.B == 13);
}

// The propagator of a reference-split step: dU = U - I stochastically rounded
// to FP32 (and its block dagger), from the field polynomial at E(t + dt/2)
// (full step, with R(E) = sum_p E^p B_p in FP64) or from the constant FP64 U.
static void reference_split_propagator(rt_ctx* c, Sys& s) {
  if (c->p.full_step) {
    PolyTerms C;
    memset(&C, 0, sizeof(C));
    const int deg2 = 2 * (c->p.taylor_terms - 1);
    for (int q = 0; q <= deg2; ++q) C.v[q] = s.Bp[q];
    const double nK = (double)nvals(s, s.pK);
    if (!r_fused(c, s))
      run(c, PC_POLY, 0, 16.0 * nK * (deg2 + 2) / 2.0, [&] {  // upper blocks: read B_0..B_deg2, write R
        launch_poly_upper(C, deg2, c->dstate, 0, s.Rm, s.pK->nnzb, s.pK->rowidx, s.pK->col, s.B, c->ws);
      });
    PolyTerms V;
    memset(&V, 0, sizeof(V));
    const int deg = c->p.taylor_terms - 1;
    for (int m = 0; m <= deg; ++m) V.v[m] = s.V[m];
    const double nU = (double)nvals(s, s.pU);
    PolyTerms32 T;
    memset(&T, 0, sizeof(T));
    const bool tail = (int)s.V32.size() == deg + 1;
    for (int m = 1; m <= deg && tail; ++m) T.v[m] = s.V32[m];
    // read V_0 (FP64) and V_1..V_deg (FP32 tail), write dU and dU^dagger
    run(c, PC_POLY, 0, 16.0 * nU + (tail ? 8.0 : 16.0) * nU * deg + 16.0 * nU, [&] {
      launch_field_poly(V, deg, c->dstate, 0, nullptr, s.dUr, s.dUHr, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B,
                        c->ws, true, s.planar, tail ? &T : nullptr);
    });
    s.u64_stale = true;
  } else {
    run(c, PC_MISC, 0, 0, [&] {
      launch_round_u_sr(s.U, s.dUr, s.dUHr, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->dstate, c->ws, s.planar);
    });
  }
}

// dK' = dK + R + M + N with M = cut(dU dK), W = dK + M, N = cut(W dU^dagger)
// (FP32 products of the small dK, every part summed in FP64); R in FP64
// (constant, or R(E) formed for this step's field by the propagator pass).
// The two products of a reference-split step for one kick slot:
//   M  = cut(dU dK) on P_M, with W = dK + M from the same epilogue;
//   dK' = dK + R + M + cut(W dU^dagger) on the upper blocks of P_K (mirrored),
//        leaving dK' rounded to FP32 for the next step's M (CUDA cores).
// 13-function blocks read the pre-transposed dagger; the 4-function kernel
// transposes while loading.
static GemmArgs m_args(Sys& s, int kick) {
  GemmArgs g = args(s.dUr, s.Kfk[kick], s.Mfk[kick]);
  g.base = s.dK[kick];
  g.U = s.Wfk[kick];
  g.add_map = s.m_to_k;
  g.a_planar = s.planar ? 1 : 0;  // dU in, W out column-planar
  return g;
}
static GemmArgs k_args(rt_ctx* c, Sys& s, int kick, int slot, bool kf_by_epilogue) {
  const bool pre_t = s.dUHr != nullptr;
  GemmArgs g = args(s.Wfk[kick], pre_t ? s.dUHr : s.dUr, s.dK[kick]);
  g.herm_max = &c->dstate->herm_bits[slot];
  g.base = s.dK[kick];
  g.addend = s.Mfk[kick];
  g.add_map = s.k_to_m;
  if (r_fused(c, s)) {
    g.rpoly = s.d_bp;
    g.rdeg = (int)s.Bp.size() - 1;
    g.poly_E = reinterpret_cast<const double*>(reinterpret_cast<const char*>(c->dstate) + offsetof(DevState, E));
  } else {
    g.base2 = s.Rm;
  }
  g.a_planar = s.planar ? 1 : 0;  // W column-planar
  g.kf32 = kf_by_epilogue ? s.Kfk[kick] : nullptr;
  return g;
}

// One kick slot, its own launches (the tensor-core products, or a context
// that does not group its products).
static void sandwich_incremental(rt_ctx* c, Sys& s, int kick, int slot) {
  TripleInfo& tM = triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);
  TripleInfo& tK = triples_for(c, s, s.pM, false, s.pU, true, s.pK, true);
  // the CUDA-core delta sandwich leaves dK' rounded to FP32 for the next step
  // (formed with dK itself); the tensor-core kernel does not, so round here
  const bool kf_by_epilogue = !tK.tiles.built;
  if (!kf_by_epilogue)
    run(c, PC_MISC, 0, 0, [&] {
      launch_d2f_pad((const double*)s.dK[kick], (float*)s.Kfk[kick], s.pK->nnzb, s.B, true, c->ws);
    });
  GemmArgs gm = m_args(s, kick);
  gm.stages = c->shape[stage_of(s.B, false)].stages;
  gm.persistent = c->shape[stage_of(s.B, false)].persistent;
  gemm(c, s, PC_UK, tM, true, true, false, false, EPI_STORE, gm, s.pM);
  const bool pre_t = s.dUHr != nullptr;
  GemmArgs gk = k_args(c, s, kick, slot, kf_by_epilogue);
  gk.stages = c->shape[stage_of(s.B, true)].stages;
  gk.persistent = c->shape[stage_of(s.B, true)].persistent;
  gemm(c, s, PC_MUDAG, tK, true, true, false, !pre_t, EPI_DELTA_SANDWICH, gk, s.pK);
}

// Grouped products: every (system, kick) pair of one block size multiplied
// by one launch per product (M, then K'), the pairs ordered by their triple
// counts, largest first, so that the launch ends on the smallest products.
// Built once, outside graph capture (the argument tables live on the device).
static bool groups_apply(const rt_ctx* c) {
  if (!incremental(c)) return false;
  for (const auto& sp : c->sys)
    if (sp->B != 13 && sp->B != 4) return false;
  return !(c->p.tensor_cores && c->p.precision == RT_FP32);
}

static void build_groups(rt_ctx* c) {
  if (c->groups_built || !groups_apply(c)) return;
  for (int st = 0; st < RT_N_STAGES; ++st) {
    const bool kstage = st & 1;
    const int B = st < 2 ? 13 : 4;
    c->groups[st] = StageGroup();
    struct Entry {
      GemmArgs g;
      int64_t triples;
      double flops, bytes;
      int sys;
    };
    std::vector<Entry> es;
    int slot = 0, si = 0;
    for (auto& sp : c->sys) {
      Sys& s = *sp;
      ++si;
      for (int k = 0; k < c->p.n_kick; ++k, ++slot) {
        if (s.B != B) continue;
        TripleInfo& ti = kstage ? triples_for(c, s, s.pM, false, s.pU, true, s.pK, true)
                                : triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);
        GemmArgs g = kstage ? prepared(c, s, ti, true, true, EPI_DELTA_SANDWICH, k_args(c, s, k, slot, true), s.pK)
                            : prepared(c, s, ti, true, true, EPI_STORE, m_args(s, k), s.pM);
        g.tri = nullptr;  // host view: not used on the device
        es.push_back({g, ti.t.n_triples, gemm_flops(ti, true), gemm_bytes(s, ti, true, true), si});
        if (kstage) {
          c->groups[st].out_bytes = std::max(c->groups[st].out_bytes, nvals(s, s.pK) * sizeof(double2));
          c->groups[st].kf_bytes = std::max(c->groups[st].kf_bytes, nvals32(s, s.pK) * sizeof(float2));
        }
      }
    }
    StageGroup& G = c->groups[st];
    const size_t ob = G.out_bytes, kb = G.kf_bytes;
    G = StageGroup();
    G.out_bytes = ob;
    G.kf_bytes = kb;
    if (es.empty()) continue;
    // systems by their triple counts, largest first; the kicks of one system
    // (the same triple list and the same dU) interleaved item by item, so that
    // their warps read each dU block at about the same time
    std::stable_sort(es.begin(), es.end(), [](const Entry& x, const Entry& y) {
      return x.triples != y.triples ? x.triples > y.triples : x.sys < y.sys;
    });
    std::vector<GemmArgs> tab;
    std::vector<int2> items;
    for (size_t i = 0; i < es.size(); ++i) {
      tab.push_back(es[i].g);
      G.flops += es[i].flops;
      G.bytes += es[i].bytes;
    }
    for (size_t i = 0; i < es.size();) {
      size_t j = i;
      while (j < es.size() && es[j].sys == es[i].sys) ++j;  // the kicks of one system
      for (int64_t it = 0; it < es[i].g.n_items; ++it)
        for (size_t e = i; e < j; ++e) items.push_back(make_int2((int)e, (int)it));
      i = j;
    }
    RT_REQUIRE(items.size() < (size_t)INT32_MAX, RT_EINVAL, "too many output blocks in one grouped product");
    if (tab.size() > 1) {
      G.d_args = c->arena.get_n<GemmArgs>(tab.size());
      G.d_items = c->arena.get_n<int2>(items.size() + 1);
      RT_CUDA_CHECK(
          cudaMemcpyAsync(G.d_args, tab.data(), sizeof(GemmArgs) * tab.size(), cudaMemcpyHostToDevice, c->ws));
      if (!items.empty())
        RT_CUDA_CHECK(
            cudaMemcpyAsync(G.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, c->ws));
      RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    }
    G.n_groups = (int)tab.size();
    G.single = tab[0];
    G.host = tab;
    G.n_items = (int64_t)items.size();
    G.B = B;
    G.planar = tab[0].a_planar;
    G.bdag = kstage && B == 4;  // the 4-function kernel transposes dU while loading
  }
  // the traces of every pair in two launches, when there are several pairs
  const int n_pairs = (int)c->sys.size() * c->p.n_kick;
  if (n_pairs > 1) {
    std::vector<TracePair> tp;
    int64_t max_nnzb = 0;
    int slot = 0;
    for (auto& sp : c->sys) {
      Sys& s = *sp;
      for (int k = 0; k < c->p.n_kick; ++k, ++slot) {
        TracePair t;
        memset(&t, 0, sizeof(t));
        t.K = s.dK[k];
        t.nnzb = s.pK->nnzb;
        t.rowidx = s.pK->rowidx;
        t.col = s.pK->col;
        t.bsize = s.d_bsize;
        t.B = s.B;
        t.S = s.S;
        t.ks_map = s.k_to_sT;
        t.Dx = s.D[0];
        t.Dy = s.D[1];
        t.Dz = s.D[2];
        t.kd_map = s.k_to_hT;
        t.herm_slot = slot;
        t.slot_index = slot;
        t.ref = s.tref;
        tp.push_back(t);
        max_nnzb = std::max<int64_t>(max_nnzb, s.pK->nnzb);
        c->tbytes += 16.0 * nvals(s, s.pK) + 8.0 * 4 * nvals(s, s.pH);
      }
    }
    c->tnb = reduce_blocks(max_nnzb);
    c->d_tpairs = c->arena.get_n<TracePair>(tp.size());
    c->tpart = c->arena.get_n<double>((size_t)tp.size() * c->tnb * 8);
    RT_CUDA_CHECK(
        cudaMemcpyAsync(c->d_tpairs, tp.data(), sizeof(TracePair) * tp.size(), cudaMemcpyHostToDevice, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    c->n_tpairs = (int)tp.size();
  }
  c->groups_built = true;
}

// The launch of one grouped stage: the launch-level arguments carry the
// tables, the item count and the launch shape; every product's own
// arguments come from its table entry.
static GemmArgs group_launch_args(const rt_ctx* c, int st, const StageGroup& G) {
  GemmArgs g;
  if (G.n_groups == 1) {
    g = G.single;
    g.wait_ns = c->wait_ns;  // the budget of this launch (a fault injection may have set it)
    g.stages = c->shape[st].stages;
    g.persistent = c->shape[st].persistent;
    return g;
  }
  memset(&g, 0, sizeof(g));
  g.grp = G.d_args;
  g.gitems = G.d_items;
  g.n_items = G.n_items;
  g.zero = c->zero32;
  g.err = c->d_err;
  g.wait_ns = c->wait_ns;
  g.a_planar = G.planar;
  g.stages = c->shape[st].stages;
  g.persistent = c->shape[st].persistent;
  return g;
}

// Launch shapes the tuner tries per stage: stages per warp (13-function
// kernel: 2 or 3) and one-shot or persistent grids.
static std::vector<LaunchShape> shape_candidates(int st) {
  if (st < 2) return {{0, 0}, {0, 1}, {3, 0}, {3, 1}};
  return {{0, 0}, {0, 1}};
}

// Times every candidate shape of every grouped stage on the context's own
// products (one warm-up launch, then `reps` launches between CUDA events) and
// keeps the fastest.  The M products write only M and W (formed again by the
// next step); the K' products write into scratch copies of their outputs, so
// the density is left as it was.
static void autotune(rt_ctx* c, int reps, std::vector<std::array<int, 4>>* rows, std::vector<double>* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RT_CUDA_CHECK(cudaEventCreate(&e0));
  RT_CUDA_CHECK(cudaEventCreate(&e1));
  try {
    for (int st = 0; st < RT_N_STAGES; ++st) {
      const StageGroup& G = c->groups[st];
      if (G.n_items == 0) continue;
      const bool kstage = st & 1;
      Scratch tmp(c);
      GemmArgs base_args = group_launch_args(c, st, G);
      if (kstage) {
        // redirect K', its FP32 copy and the hermiticity record to scratch
        double2* kout = tmp.get_n<double2>(G.out_bytes / sizeof(double2) + 1);
        float2* fout = tmp.get_n<float2>(G.kf_bytes / sizeof(float2) + 1);
        unsigned long long* hm = tmp.get_n<unsigned long long>(1);
        std::vector<GemmArgs> tab = G.host;
        for (GemmArgs& a : tab) {
          a.C = kout;
          a.kf32 = fout;
          a.herm_max = hm;
        }
        if (G.n_groups == 1) {
          base_args.C = kout;
          base_args.kf32 = fout;
          base_args.herm_max = hm;
        } else {
          GemmArgs* d_tab = tmp.get_n<GemmArgs>(tab.size());
          RT_CUDA_CHECK(
              cudaMemcpyAsync(d_tab, tab.data(), sizeof(GemmArgs) * tab.size(), cudaMemcpyHostToDevice, c->ws));
          base_args.grp = d_tab;
        }
      }
      double best = 1e300;
      LaunchShape pick = c->shape[st];
      for (const LaunchShape& sh : shape_candidates(st)) {
        GemmArgs g = base_args;
        g.stages = sh.stages;
        g.persistent = sh.persistent;
        auto launch = [&] {
          launch_gemm(G.B, true, true, false, G.bdag, kstage ? EPI_DELTA_SANDWICH : EPI_STORE, g, c->ws);
        };
        launch();
        RT_CUDA_CHECK(cudaEventRecord(e0, c->ws));
        for (int r = 0; r < reps; ++r) launch();
        RT_CUDA_CHECK(cudaEventRecord(e1, c->ws));
        RT_CUDA_CHECK(cudaEventSynchronize(e1));
        float t = 0.f;
        RT_CUDA_CHECK(cudaEventElapsedTime(&t, e0, e1));
        const double per = (double)t / reps;
        if (rows) rows->push_back({st, sh.stages == 0 ? 2 : sh.stages, sh.persistent, 0});
        if (ms) ms->push_back(per);
        if (per < best) {
          best = per;
          pick = sh;
        }
      }
      c->shape[st] = pick;
      if (rows)
        for (auto& r : *rows)
          if (r[0] == st) r[3] = (r[1] == (pick.stages == 0 ? 2 : pick.stages) && r[2] == pick.persistent) ? 1 : 0;
      ::check_device_error(c);
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->graph_dirty = true;
}

static void grouped_stage(rt_ctx* c, int st) {
  const StageGroup& G = c->groups[st];
  if (G.n_items == 0) return;
  const bool kstage = st & 1;
  GemmArgs g = group_launch_args(c, st, G);
  run(c, kstage ? PC_MUDAG : PC_UK, G.flops, G.bytes, [&] {
    launch_gemm(G.B, true, true, false, G.bdag, kstage ? EPI_DELTA_SANDWICH : EPI_STORE, g, c->ws);
  });
}

static void enqueue_step(rt_ctx* c) {
  run(c, PC_MISC, 0, 0, [&] { launch_begin_step(c->dstate, c->field, c->p.dt, c->n_slots, c->ws); });
  int slot = 0;
  const bool grouped = c->groups_built;
  for (auto& sp : c->sys) {
    Sys& s = *sp;
    if (incremental(c)) reference_split_propagator(c, s);
    else if (c->p.full_step) build_propagator(c, s, c->p.precision == RT_FP32);
    for (int k = 0; k < c->p.n_kick && !grouped; ++k) {
      if (incremental(c)) sandwich_incremental(c, s, k, slot + k);
      else sandwich(c, s, k, slot + k);
    }
    slot += c->p.n_kick;
  }
  if (grouped)
    for (int st : {0, 2, 1, 3}) grouped_stage(c, st);  // every M product, then every K' product
  run(c, PC_MISC, 0, 0, [&] { launch_end_step(c->dstate, c->p.dt, c->ws); });
  if (grouped && c->n_tpairs > 1) {
    run(
        c, PC_OBS, 0, c->tbytes,
        [&] {
          launch_traces_grouped(c->d_tpairs, c->n_tpairs, c->tnb, c->tpart, c->dstate, c->ring, c->p.obs_capacity,
                                c->n_slots, c->ws);
        },
        2);
    return;
  }
  slot = 0;
  for (auto& sp : c->sys) {
    for (int k = 0; k < c->p.n_kick; ++k) observe(c, *sp, k, slot + k);
    slot += c->p.n_kick;
  }
}

// ----------------------------------------------------------------------------
// set-up helpers used by the API
// ----------------------------------------------------------------------------
static void reset_time(rt_ctx* c) {
  DevState z;
  memset(&z, 0, sizeof(z));
  RT_CUDA_CHECK(cudaMemcpyAsync(c->dstate, &z, sizeof(DevState), cudaMemcpyHostToDevice, c->ws));
  c->host_step = 0;
  c->t_host = 0.0;
  std::fill(c->read_upto.begin(), c->read_upto.end(), 0);
}

// K <- V K V^dagger with V = exp(+i kappa S^-1 D_dir) (Taylor, powers cut to r_U)
static void kick_one(rt_ctx* c, Sys& s, int kick, int dir, double kappa) {
  TripleInfo& tT = triples_for(c, s, s.pSinv, false, s.pH, false, s.pT, false);
  gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.D[dir], s.T), s.pT);
  taylor_series(c, s, s.T, -kappa, c->p.kick_terms, false);
  TripleInfo& tM = triples_for(c, s, s.pU, false, s.pK, false, s.pM, false);
  TripleInfo& tK = triples_for(c, s, s.pM, false, s.pU, true, s.pK, true);
  gemm(c, s, PC_MISC, tM, false, true, false, false, EPI_STORE, args(s.U, s.K[kick], s.M), s.pM);
  gemm(c, s, PC_MISC, tK, false, true, false, true, EPI_SANDWICH, args(s.M, s.U, s.K[kick]), s.pK);
  s.u_ready = false;  // U now holds V
  s.duf_current = false;
}

// K0 = f(S^-1 H0) S^-1 by a Chebyshev expansion (real FP64 on P_K)
static void ground_state(rt_ctx* c, Sys& s, int order, double mu, double kT, double e_lo, double e_hi) {
  RT_REQUIRE(order >= 0 && kT > 0 && e_hi > e_lo, RT_EINVAL, "bad ground-state parameters");
  Pattern* PK = s.pK;
  TripleInfo& tT = triples_for(c, s, s.pSinv, false, s.pH, false, s.pT, false);
  TripleInfo& tTK = triples_for(c, s, s.pT, false, PK, false, PK, false);
  gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.H0, s.T), s.pT);
  // Chebyshev coefficients of the Fermi function (Chebyshev-Gauss quadrature)
  const double a = 0.5 * (e_hi + e_lo), w = 0.5 * (e_hi - e_lo);
  const int Mq = 4 * (order + 1);
  std::vector<double> f(Mq), th(Mq), coef(order + 1);
  for (int k = 0; k < Mq; ++k) {
    th[k] = M_PI * (k + 0.5) / Mq;
    double e = a + w * std::cos(th[k]);
    f[k] = 0.5 * (1.0 - std::tanh(0.5 * (e - mu) / kT));
  }
  for (int n = 0; n <= order; ++n) {
    double acc = 0.0;
    for (int k = 0; k < Mq; ++k) acc += f[k] * std::cos(n * th[k]);
    coef[n] = (n ? 2.0 : 1.0) / Mq * acc;
  }
  size_t nv = nvals(s, PK);
  double* Y0 = c->arena.get_n<double>(nv);
  double* Y1 = c->arena.get_n<double>(nv);
  double* Y2 = c->arena.get_n<double>(nv);
  double* TY = c->arena.get_n<double>(nv);
  double* Kr = c->arena.get_n<double>(nv);
  launch_restrict(s.Sinv, Y0, s.k_to_sinv, PK->nnzb, s.B, 0, c->ws);
  RT_CUDA_CHECK(cudaMemcpyAsync(Kr, Y0, sizeof(double) * nv, cudaMemcpyDeviceToDevice, c->ws));
  launch_scale(Kr, coef[0], (int64_t)nv, c->ws);
  double *Ym = Y0, *Yc = Y0, *Yn = Y1;
  for (int n = 1; n <= order; ++n) {
    gemm(c, s, PC_MISC, tTK, false, false, false, false, EPI_STORE, args(s.T, Yc, TY), PK);
    launch_cheb_step(TY, Yc, Ym, Yn, Kr, a, w, coef[n], n == 1 ? 1 : 0, (int64_t)nv, c->ws);
    // rotate: (Ym, Yc) <- (Yc, Yn); Yn <- a free buffer
    double* freeb = (n == 1) ? Y2 : Ym;
    Ym = Yc;
    Yc = Yn;
    Yn = freeb;
  }
  for (size_t k = 0; k < s.K.size(); ++k)
    launch_symmetrise_to_complex(Kr, s.K[k], PK->nnzb, PK->rowidx, PK->col, PK->tmap, s.d_bsize, s.B, c->ws);
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
}

static void ensure_unitarity_lists(rt_ctx* c, Sys& s) {
  if (s.pW) return;
  double rW = c->p.r_U + std::max(s.r_S, 1e-9);
  s.pW = pattern_for(c, s, rW);
  s.Sc = c->arena.get_n<double2>(nvals(s, s.pS));
  int32_t* ident = c->arena.get_n<int32_t>(s.pS->nnzb);
  std::vector<int32_t> h(s.pS->nnzb);
  for (int64_t q = 0; q < s.pS->nnzb; ++q) h[q] = (int32_t)q;
  RT_CUDA_CHECK(cudaMemcpyAsync(ident, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, c->ws));
  launch_restrict(s.S, (double*)s.Sc, ident, s.pS->nnzb, s.B, 1, c->ws);
  s.W = c->arena.get_n<double2>(nvals(s, s.pW));
  s.E = c->arena.get_n<double2>(nvals(s, s.pU));
  s.u_to_s = block_map(c, s.pU, s.pS, false);
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
}

static void unitarity(rt_ctx* c, Sys& s, int metric, double* mx, double* mean) {
  ensure_unitarity_lists(c, s);
  refresh_u64(c, s);
  if (s.duf_current)
    launch_u_from_delta(s.dUf, s.U, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws);  // U = I + dU
  if (metric) {
    TripleInfo& tW = triples_for(c, s, s.pS, false, s.pU, false, s.pW, false);
    TripleInfo& tE = triples_for(c, s, s.pU, true, s.pW, false, s.pU, false);
    gemm(c, s, PC_MISC, tW, false, true, false, false, EPI_STORE, args(s.Sc, s.U, s.W), s.pW);
    gemm(c, s, PC_MISC, tE, false, true, true, false, EPI_STORE, args(s.U, s.W, s.E), s.pU);
  } else {
    TripleInfo& tE = triples_for(c, s, s.pU, true, s.pU, false, s.pU, false);
    gemm(c, s, PC_MISC, tE, false, true, true, false, EPI_STORE, args(s.U, s.U, s.E), s.pU);
  }
  double* pmax = c->arena.get_n<double>(1024);
  double* psum = c->arena.get_n<double>(1024);
  int nb = launch_unitarity_dev(s.E, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.d_bsize, s.B, metric ? s.S : nullptr,
                                metric ? s.u_to_s : nullptr, pmax, psum, c->ws);
  std::vector<double> hm(nb), hs(nb);
  RT_CUDA_CHECK(cudaMemcpyAsync(hm.data(), pmax, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->ws));
  RT_CUDA_CHECK(cudaMemcpyAsync(hs.data(), psum, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->ws));
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
  double m = 0.0, sm = 0.0;
  for (int i = 0; i < nb; ++i) {
    m = std::max(m, hm[i]);
    sm += hs[i];
  }
  int64_t cnt = 0;
  for (int i = 0; i < s.n_atoms; ++i)
    for (int q = s.pU->h_rowptr[i]; q < s.pU->h_rowptr[i + 1]; ++q)
      cnt += (int64_t)s.bsize[i] * s.bsize[s.pU->h_col[q]];
  *mx = m;
  *mean = cnt ? sm / (double)cnt : 0.0;
}

static Pattern* pattern_by_id(Sys& s, int which) {
  switch (which) {
    case RT_PAT_S: return s.pS;
    case RT_PAT_H: return s.pH;
    case RT_PAT_SINV: return s.pSinv;
    case RT_PAT_T: return s.pT;
    case RT_PAT_U: return s.pU;
    case RT_PAT_K: return s.pK;
    case RT_PAT_M: return s.pM;
    case RT_PAT_A: return s.pA;
    case RT_PAT_W: return s.pW;
    default: return nullptr;
  }
}

// (pattern, device values, complex?) of a readable matrix
static void matrix_by_id(rt_ctx* c, Sys& s, int kick, int which, Pattern** P, const void** v, bool* cplx) {
  *cplx = false;
  switch (which) {
    case RT_MAT_S: *P = s.pS; *v = s.S; return;
    case RT_MAT_H0: *P = s.pH; *v = s.H0; return;
    case RT_MAT_DX: *P = s.pH; *v = s.D[0]; return;
    case RT_MAT_DY: *P = s.pH; *v = s.D[1]; return;
    case RT_MAT_DZ: *P = s.pH; *v = s.D[2]; return;
    case RT_MAT_SINV: *P = s.pSinv; *v = s.Sinv; return;
    case RT_MAT_T: *P = s.pT; *v = s.T; return;
    case RT_MAT_U: *P = s.pU; *v = s.U; *cplx = true; return;
    case RT_MAT_K:
      RT_REQUIRE(kick >= 0 && kick < c->p.n_kick, RT_EINVAL, "kick index out of range");
      *P = s.pK; *v = s.K[kick]; *cplx = true; return;
    case RT_MAT_X:
      RT_REQUIRE(s.X != nullptr, RT_EINVAL, "X exists only in the Crank-Nicolson mode");
      *P = s.pU; *v = s.X; *cplx = true; return;
    default: throw Error{RT_EINVAL, "unknown matrix id"};
  }
}

static int64_t true_elems(const Sys& s, const Pattern* P) {
  int64_t n = 0;
  for (int i = 0; i < s.n_atoms; ++i)
    for (int q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) n += (int64_t)s.bsize[i] * s.bsize[P->h_col[q]];
  return n;
}

}  // namespace rt

// ============================================================================
// C ABI
// ============================================================================
using namespace rt;

template <class F>
static rt_status guarded(rt_ctx* c, F&& f) {
  if (!c) return RT_EINVAL;
  if (c->poisoned) return RT_ESTATE;
  c->err.clear();
  try {
    RT_CUDA_CHECK(cudaEventRecord(c->ev_in, c->user));
    RT_CUDA_CHECK(cudaStreamWaitEvent(c->ws, c->ev_in, 0));
    rt_status st = f();
    RT_CUDA_CHECK(cudaEventRecord(c->ev_out, c->ws));
    RT_CUDA_CHECK(cudaStreamWaitEvent(c->user, c->ev_out, 0));
    return st;
  } catch (const Error& e) {
    c->err = e.msg;
    if (e.code == RT_ECUDA || e.code == RT_ETIMEOUT || e.code == RT_EINTERNAL) c->poisoned = true;
    return e.code;
  } catch (const std::exception& e) {
    c->err = e.what();
    c->poisoned = true;
    return RT_EINTERNAL;
  }
}

// Raises RT_ETIMEOUT when a kernel recorded that a bounded wait gave up.  Code
// 2 (the drain of the copies in flight ran out as well) also marks the context
// unrecoverable: no checkpoint restore is accepted after it.
static void check_device_error(rt_ctx* c) {
  int e = 0;
  RT_CUDA_CHECK(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->ws));
  RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
  if (e >= 2) c->unrecoverable = true;
  if (e) throw Error{RT_ETIMEOUT, "a device-side bounded wait gave up (error word " + std::to_string(e) + ")"};
}

static rt_status check_sys(rt_ctx* c, int32_t sys) {
  if (sys < 0 || sys >= (int32_t)c->sys.size()) throw Error{RT_EINVAL, "system index out of range"};
  return RT_OK;
}

extern "C" {

rt_status rt_default_params(rt_params* p) {
  if (!p) return RT_EINVAL;
  memset(p, 0, sizeof(*p));
  p->r_Sinv = p->r_T = p->r_U = p->r_K = p->r_M = 8.0;
  p->dt = 0.05;
  p->prop = RT_PROP_EM;
  p->taylor_terms = 6;
  p->hot_tol = 1e-10;
  p->hot_maxit = 100;
  p->hot_step_iters = 2;
  p->hot_fp64_iters = 1;
  p->tensor_cores = 0;
  p->packed_fma = 1;
  p->precision = RT_FP64;
  p->full_step = 1;
  p->n_kick = 1;
  p->kick_terms = 12;
  p->obs_capacity = 4096;
  p->use_graph = 1;
  return RT_OK;
}

rt_status rt_create(rt_ctx** out, const rt_system* sys, int32_t n_sys, const rt_params* p, void* cuda_stream,
                    rt_alloc_fn alloc, rt_free_fn free_fn, void* alloc_user) {
  if (!out) return RT_EINVAL;
  *out = nullptr;
  auto* c = new rt_ctx();
  c->alloc.alloc = alloc;
  c->alloc.free = free_fn;
  c->alloc.user = alloc_user;
  c->arena.alloc = &c->alloc;
  c->user = (cudaStream_t)cuda_stream;
  try {
    RT_REQUIRE(sys && n_sys > 0 && p, RT_EINVAL, "need at least one system and params");
    c->p = *p;
    const rt_params& q = c->p;
    RT_REQUIRE(q.r_Sinv > 0 && q.r_T > 0 && q.r_U > 0 && q.r_K > 0 && q.r_M > 0, RT_EINVAL, "radii must be positive");
    RT_REQUIRE(q.dt > 0 && std::isfinite(q.dt), RT_EINVAL, "dt must be positive");
    RT_REQUIRE(q.prop >= RT_PROP_EM && q.prop <= RT_PROP_M4, RT_EINVAL,
               "prop must be RT_PROP_EM, RT_PROP_CN, RT_PROP_ETRS or RT_PROP_M4");
    RT_REQUIRE(q.taylor_terms >= 1 && q.taylor_terms <= 32, RT_EINVAL, "taylor_terms must be in 1..32");
    RT_REQUIRE(q.precision == RT_FP64 || q.precision == RT_FP32, RT_EINVAL, "precision must be RT_FP64 or RT_FP32");
    RT_REQUIRE(q.n_kick >= 1 && q.n_kick <= 3, RT_EINVAL, "n_kick must be in 1..3");
    RT_REQUIRE(q.obs_capacity >= 1, RT_EINVAL, "obs_capacity must be positive");
    RT_REQUIRE(q.hot_step_iters >= 0 && q.hot_maxit >= 0 && q.kick_terms >= 1, RT_EINVAL, "bad iteration counts");
    RT_REQUIRE(q.hot_step_iters == 0 || (q.hot_fp64_iters >= 1 && q.hot_fp64_iters <= q.hot_step_iters), RT_EINVAL,
               "hot_fp64_iters must be in 1..hot_step_iters");
    RT_REQUIRE((int64_t)n_sys * q.n_kick <= RT_MAX_SLOTS, RT_EINVAL, "too many (system, kick) pairs");
    RT_REQUIRE(!q.incremental || q.precision == RT_FP32, RT_EINVAL, "the reference split needs precision RT_FP32");
    RT_REQUIRE(!q.incremental || !q.full_step || (q.field_poly && q.prop == RT_PROP_EM), RT_EINVAL,
               "the reference split with full_step = 1 needs the EM field polynomial (field_poly = 1)");
    RT_CUDA_CHECK(cudaStreamCreateWithFlags(&c->ws, cudaStreamNonBlocking));
    RT_CUDA_CHECK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    RT_CUDA_CHECK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    c->arena.stream = c->ws;
    RT_CUDA_CHECK(cudaEventRecord(c->ev_in, c->user));
    RT_CUDA_CHECK(cudaStreamWaitEvent(c->ws, c->ev_in, 0));
    c->n_slots = n_sys * q.n_kick;
    c->read_upto.assign(c->n_slots, 0);
    c->dstate = c->arena.get_n<DevState>(1);
    c->zero32 = c->arena.get(13 * 16 * sizeof(float2));
    RT_CUDA_CHECK(cudaMemsetAsync(c->zero32, 0, 13 * 16 * sizeof(float2), c->ws));
    c->d_err = c->arena.get_n<int>(1);
    RT_CUDA_CHECK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->ws));
    c->ring = c->arena.get_n<double>((size_t)q.obs_capacity * c->n_slots * RT_NOBS);
    RT_CUDA_CHECK(cudaMemsetAsync(c->ring, 0, sizeof(double) * (size_t)q.obs_capacity * c->n_slots * RT_NOBS, c->ws));
    reset_time(c);
    for (int i = 0; i < n_sys; ++i) {
      c->sys.push_back(std::make_unique<Sys>());
      setup_system(c, *c->sys.back(), sys[i]);
    }
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
  } catch (const Error& e) {
    if (c->ws) cudaStreamSynchronize(c->ws);
    c->arena.release_all();
    if (c->ws) cudaStreamDestroy(c->ws);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    rt_status code = e.code;
    // keep the message reachable through a static buffer for the failed create
    static thread_local std::string last;
    last = e.msg;
    fprintf(stderr, "rt_create: %s\n", e.msg.c_str());
    delete c;
    return code;
  }
  *out = c;
  return RT_OK;
}

rt_status rt_set_field(rt_ctx* c, const rt_field* f) {
  return guarded(c, [&] {
    RT_REQUIRE(f, RT_EINVAL, "NULL field");
    RT_REQUIRE(f->dir >= 0 && f->dir < 3, RT_EINVAL, "field dir must be 0, 1 or 2");
    RT_REQUIRE(f->kind >= RT_FIELD_NONE && f->kind <= RT_FIELD_CONSTANT, RT_EINVAL, "unknown field kind");
    if (f->kind == RT_FIELD_GAUSSIAN) RT_REQUIRE(f->sigma > 0, RT_EINVAL, "sigma must be positive");
    bool dir_changed = f->dir != c->field.dir;
    c->field.kind = f->kind;
    c->field.dir = f->dir;
    c->field.E0 = f->E0;
    c->field.t0 = f->t0;
    c->field.sigma = f->sigma;
    c->field.omega = f->omega;
    c->graph_dirty = true;
    if (dir_changed && c->p.precision == RT_FP32 && c->p.prop != RT_PROP_CN) {
      for (auto& sp : c->sys) {
        Sys& s = *sp;
        if (!s.sinv_ready) continue;
        TripleInfo& tT = triples_for(c, s, s.pSinv, false, s.pH, false, s.pT, false);
        gemm(c, s, PC_MISC, tT, false, false, false, false, EPI_STORE, args(s.Sinv, s.D[c->field.dir], s.TD), s.pT);
      }
    }
    if (dir_changed && c->p.field_poly)
      for (auto& sp : c->sys)
        if (sp->sinv_ready) build_field_poly(c, *sp);
    return RT_OK;
  });
}

rt_status rt_inverse(rt_ctx* c, int32_t sys, int32_t* iters, double* residual) {
  return guarded(c, [&] {
    if (sys >= 0) check_sys(c, sys);
    rt_status worst = RT_OK;
    const int32_t maxit = c->p.hot_maxit;
    if (c->inject & RT_FAULT_HOTELLING_MAXITER1) {
      c->p.hot_maxit = 1;
      c->inject &= ~(uint32_t)RT_FAULT_HOTELLING_MAXITER1;
    }
    for (size_t i = 0; i < c->sys.size(); ++i) {
      rt_status st = RT_OK;
      try {
        st = hotelling_sinv(c, *c->sys[i]);
      } catch (...) {
        c->p.hot_maxit = maxit;
        throw;
      }
      if (st != RT_OK) {
        worst = st;
        c->err = "Hotelling " + c->sys[i]->sinv_status + " for system " + std::to_string(i) +
                 " (residual " + std::to_string(c->sys[i]->sinv_resid) + ")";
      }
    }
    c->p.hot_maxit = maxit;
    int32_t k = sys >= 0 ? sys : 0;
    if (iters) *iters = c->sys[k]->sinv_iters;
    if (residual) *residual = c->sys[k]->sinv_resid;
    return worst;
  });
}

rt_status rt_set_density(rt_ctx* c, int32_t sys, int32_t kick, const double* h) {
  return guarded(c, [&] {
    check_sys(c, sys);
    RT_REQUIRE(kick >= 0 && kick < c->p.n_kick, RT_EINVAL, "kick index out of range");
    RT_REQUIRE(h, RT_EINVAL, "NULL density");
    Sys& s = *c->sys[sys];
    const Pattern& P = *s.pK;
    const int B = s.B;
    // K replaced: it is the density again; the reference split keeps K_ref and
    // carries the new K as dK = K - K_ref from the next step
    if (!s.dk_fresh.empty()) s.dk_fresh[kick] = 0;
    if (s.n_true == (int64_t)s.n_atoms * B) {
      // no padded atoms: the caller's layout is the device layout; copy directly
      // (a DMA at full speed when the caller's buffer is pinned)
      RT_CUDA_CHECK(cudaMemcpyAsync(s.K[kick], h, sizeof(double2) * nvals(s, s.pK), cudaMemcpyHostToDevice, c->ws));
      reset_time(c);
      RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
      return RT_OK;
    }
    std::vector<double> buf(2 * (size_t)P.nnzb * B * B, 0.0);
    size_t o = 0;
    for (int i = 0; i < s.n_atoms; ++i)
      for (int q = P.h_rowptr[i]; q < P.h_rowptr[i + 1]; ++q) {
        int j = P.h_col[q];
        int bi = s.bsize[i], bj = s.bsize[j];
        double* blk = buf.data() + 2 * (size_t)q * B * B;
        for (int a = 0; a < bi; ++a)
          for (int b = 0; b < bj; ++b) {
            blk[2 * (a * B + b)] = h[2 * (o + (size_t)a * bj + b)];
            blk[2 * (a * B + b) + 1] = h[2 * (o + (size_t)a * bj + b) + 1];
          }
        o += (size_t)bi * bj;
      }
    RT_CUDA_CHECK(cudaMemcpyAsync(s.K[kick], buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, c->ws));
    reset_time(c);
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    return RT_OK;
  });
}

rt_status rt_ground_state(rt_ctx* c, int32_t sys, int32_t order, double mu, double kT, double e_lo, double e_hi) {
  return guarded(c, [&] {
    check_sys(c, sys);
    Sys& s = *c->sys[sys];
    RT_REQUIRE(s.sinv_ready, RT_ESTATE, "call rt_inverse first");
    std::fill(s.dk_fresh.begin(), s.dk_fresh.end(), 0);  // every K replaced, the reference too
    s.ref_ready = false;
    ground_state(c, s, order, mu, kT, e_lo, e_hi);
    reset_time(c);
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    return RT_OK;
  });
}

rt_status rt_kick(rt_ctx* c, int32_t sys, int32_t kick, int32_t dir, double kappa) {
  return guarded(c, [&] {
    check_sys(c, sys);
    RT_REQUIRE(kick >= 0 && kick < c->p.n_kick, RT_EINVAL, "kick index out of range");
    RT_REQUIRE(dir >= 0 && dir < 3, RT_EINVAL, "dir must be 0, 1 or 2");
    RT_REQUIRE(std::isfinite(kappa), RT_EINVAL, "kappa must be finite");
    Sys& s = *c->sys[sys];
    RT_REQUIRE(s.sinv_ready, RT_ESTATE, "call rt_inverse first");
    materialize(c, s);
    kick_one(c, s, kick, dir, kappa);
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    return RT_OK;
  });
}

rt_status rt_propagator(rt_ctx* c, double t) {
  return guarded(c, [&] {
    for (auto& sp : c->sys) RT_REQUIRE(sp->sinv_ready, RT_ESTATE, "call rt_inverse first");
    // field at t + dt/2 through the device state
    DevState tmp;
    RT_CUDA_CHECK(cudaMemcpyAsync(&tmp, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    double t_saved = tmp.t;
    tmp.t = t;
    RT_CUDA_CHECK(cudaMemcpyAsync(c->dstate, &tmp, sizeof(DevState), cudaMemcpyHostToDevice, c->ws));
    launch_begin_step(c->dstate, c->field, c->p.dt, c->n_slots, c->ws);
    for (auto& sp : c->sys) {
      Sys& s = *sp;
      if (incremental(c)) {
        // the propagator is built in FP64; each step rounds it to FP32
        // stochastically.  With a constant U the reference part R depends on
        // U, so a new U drops the reference; with the field polynomial it does not.
        build_propagator(c, s, false);
        if (!c->p.full_step) s.r_ready = false;
        s.u64_stale = false;
      } else {
        build_propagator(c, s, c->p.precision == RT_FP32);
      }
      s.u_ready = true;
    }
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    RT_CUDA_CHECK(cudaMemcpyAsync(&tmp, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    tmp.t = t_saved;
    RT_CUDA_CHECK(cudaMemcpyAsync(c->dstate, &tmp, sizeof(DevState), cudaMemcpyHostToDevice, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    c->graph_dirty = true;
    return RT_OK;
  });
}

rt_status rt_autotune(rt_ctx* c, int32_t reps, int32_t max_rows, int32_t* n_rows, int32_t* rows, double* ms) {
  return guarded(c, [&] {
    RT_REQUIRE(reps >= 1 && reps <= 100, RT_EINVAL, "reps must be 1..100");
    RT_REQUIRE(max_rows >= 0 && (max_rows == 0 || (rows && ms)), RT_EINVAL, "bad output buffers");
    RT_REQUIRE(groups_apply(c), RT_ESTATE,
               "the tuner times the reference split's CUDA-core products (incremental = 1, tensor_cores = 0, "
               "block sizes 4 and 13)");
    build_groups(c);
    std::vector<std::array<int, 4>> r;
    std::vector<double> t;
    autotune(c, reps, &r, &t);
    if (n_rows) *n_rows = (int32_t)r.size();
    for (size_t i = 0; i < r.size() && (int32_t)i < max_rows; ++i) {
      for (int k = 0; k < 4; ++k) rows[4 * i + k] = r[i][k];
      ms[i] = t[i];
    }
    return RT_OK;
  });
}

rt_status rt_set_launch_shape(rt_ctx* c, int32_t stage, int32_t stages, int32_t persistent) {
  return guarded(c, [&] {
    RT_REQUIRE(stage >= 0 && stage < RT_N_STAGES, RT_EINVAL, "stage must be 0..3");
    RT_REQUIRE(stages == 2 || (stages == 3 && stage < 2), RT_EINVAL,
               "stages per warp: 2, or 3 for the 13-function stages");
    RT_REQUIRE(persistent == 0 || persistent == 1, RT_EINVAL, "persistent must be 0 or 1");
    c->shape[stage].stages = stages == 2 ? 0 : stages;
    c->shape[stage].persistent = persistent;
    c->graph_dirty = true;
    return RT_OK;
  });
}

rt_status rt_get_launch_shape(rt_ctx* c, int32_t stage, int32_t* stages, int32_t* persistent) {
  return guarded(c, [&] {
    RT_REQUIRE(stage >= 0 && stage < RT_N_STAGES, RT_EINVAL, "stage must be 0..3");
    RT_REQUIRE(stages && persistent, RT_EINVAL, "NULL output");
    *stages = c->shape[stage].stages == 0 ? 2 : c->shape[stage].stages;
    *persistent = c->shape[stage].persistent;
    return RT_OK;
  });
}

rt_status rt_step(rt_ctx* c, int32_t n) {
  return guarded(c, [&] {
    RT_REQUIRE(n >= 0, RT_EINVAL, "n must be non-negative");
    for (auto& sp : c->sys) {
      RT_REQUIRE(sp->sinv_ready, RT_ESTATE, "call rt_inverse first");
      if (!c->p.full_step) RT_REQUIRE(sp->u_ready, RT_ESTATE, "call rt_propagator first (full_step = 0)");
    }
    if (n == 0) return RT_OK;
    if (incremental(c))
      for (auto& sp : c->sys) prepare_reference(c, *sp);
    build_groups(c);
    if (c->inject & RT_FAULT_WAIT_TIMEOUT_0) {
      // one step, launched directly, with a zero wait budget; the error word
      // is read back here so that this call reports the expiry
      c->inject &= ~(uint32_t)RT_FAULT_WAIT_TIMEOUT_0;
      c->wait_ns = 0;
      try {
        enqueue_step(c);
      } catch (...) {
        c->wait_ns = 2000000000ll;
        throw;
      }
      c->wait_ns = 2000000000ll;
      c->graph_dirty = true;
      c->host_step += 1;
      c->t_host += c->p.dt;
      RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
      check_device_error(c);
      if (n == 1) return RT_OK;
      --n;
    }
    if (c->profiling || !c->p.use_graph) {
      for (int i = 0; i < n; ++i) enqueue_step(c);
      if (c->profiling) collect_profile(c);
    } else {
      if (c->graph_dirty || !c->gexec) {
        if (c->gexec) {
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        RT_CUDA_CHECK(cudaStreamBeginCapture(c->ws, cudaStreamCaptureModeThreadLocal));
        try {
          enqueue_step(c);
        } catch (...) {
          cudaStreamEndCapture(c->ws, &graph);
          if (graph) cudaGraphDestroy(graph);
          throw;
        }
        RT_CUDA_CHECK(cudaStreamEndCapture(c->ws, &graph));
        cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        RT_CUDA_CHECK(e);
        c->graph_dirty = false;
      }
      for (int i = 0; i < n; ++i) RT_CUDA_CHECK(cudaGraphLaunch(c->gexec, c->ws));
    }
    c->host_step += n;
    c->t_host += n * c->p.dt;
    return RT_OK;
  });
}

rt_status rt_observables(rt_ctx* c, int32_t sys, int32_t kick, double* out, int32_t max_steps, int32_t* n_out) {
  return guarded(c, [&] {
    check_sys(c, sys);
    RT_REQUIRE(kick >= 0 && kick < c->p.n_kick, RT_EINVAL, "kick index out of range");
    RT_REQUIRE(out && n_out && max_steps >= 0, RT_EINVAL, "bad output buffer");
    int slot = sys * c->p.n_kick + kick;
    int64_t cap = c->p.obs_capacity;
    int64_t first = std::max(c->read_upto[slot], c->host_step - cap);
    int64_t cnt = std::min<int64_t>(c->host_step - first, max_steps);
    std::vector<double> ring((size_t)cap * c->n_slots * RT_NOBS);
    RT_CUDA_CHECK(cudaMemcpyAsync(ring.data(), c->ring, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    check_device_error(c);
    bool bad = false;
    for (int64_t k = 0; k < cnt; ++k) {
      int64_t r = (first + k) % cap;
      const double* rec = ring.data() + (r * c->n_slots + slot) * RT_NOBS;
      for (int v = 0; v < RT_NOBS; ++v) {
        out[k * RT_NOBS + v] = rec[v];
        if (!std::isfinite(rec[v])) bad = true;
      }
    }
    c->read_upto[slot] = first + cnt;
    *n_out = (int32_t)cnt;
    if (bad) {
      c->err = "NaN/Inf in an observable";
      return RT_ENUMERIC;
    }
    return RT_OK;
  });
}

rt_status rt_pattern_size(rt_ctx* c, int32_t sys, int32_t which, int64_t* nnzb) {
  return guarded(c, [&] {
    check_sys(c, sys);
    Sys& s = *c->sys[sys];
    if (which == RT_PAT_W) ensure_unitarity_lists(c, s);
    Pattern* P = pattern_by_id(s, which);
    RT_REQUIRE(P && nnzb, RT_EINVAL, "unknown pattern id");
    *nnzb = P->nnzb;
    return RT_OK;
  });
}

rt_status rt_get_pattern(rt_ctx* c, int32_t sys, int32_t which, int32_t* rowptr, int32_t* col) {
  return guarded(c, [&] {
    check_sys(c, sys);
    Sys& s = *c->sys[sys];
    if (which == RT_PAT_W) ensure_unitarity_lists(c, s);
    Pattern* P = pattern_by_id(s, which);
    RT_REQUIRE(P && rowptr && col, RT_EINVAL, "unknown pattern id or NULL output");
    std::memcpy(rowptr, P->h_rowptr.data(), sizeof(int32_t) * (s.n_atoms + 1));
    if (P->nnzb) std::memcpy(col, P->h_col.data(), sizeof(int32_t) * P->nnzb);
    return RT_OK;
  });
}

rt_status rt_matrix_size(rt_ctx* c, int32_t sys, int32_t which, int64_t* n) {
  return guarded(c, [&] {
    check_sys(c, sys);
    Sys& s = *c->sys[sys];
    Pattern* P;
    const void* v;
    bool cplx;
    matrix_by_id(c, s, 0, which, &P, &v, &cplx);
    RT_REQUIRE(n, RT_EINVAL, "NULL output");
    *n = 2 * true_elems(s, P);
    return RT_OK;
  });
}

rt_status rt_get_matrix(rt_ctx* c, int32_t sys, int32_t kick, int32_t which, double* vals, int64_t capacity) {
  return guarded(c, [&] {
    check_sys(c, sys);
    Sys& s = *c->sys[sys];
    Pattern* P;
    const void* v;
    bool cplx;
    if (which == RT_MAT_K) materialize(c, s, true);
    if (which == RT_MAT_U) refresh_u64(c, s);
    if (which == RT_MAT_U && s.duf_current)
      launch_u_from_delta(s.dUf, s.U, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws);  // U = I + (U - I)
    matrix_by_id(c, s, kick, which, &P, &v, &cplx);
    RT_REQUIRE(vals, RT_EINVAL, "NULL output");
    int64_t need = 2 * true_elems(s, P);
    RT_REQUIRE(capacity >= need, RT_EINVAL, "output buffer too small");
    const int B = s.B;
    size_t nv = (size_t)P->nnzb * B * B * (cplx ? 2 : 1);
    std::vector<double> buf(nv);
    if (nv) RT_CUDA_CHECK(cudaMemcpyAsync(buf.data(), v, sizeof(double) * nv, cudaMemcpyDeviceToHost, c->ws));
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    size_t o = 0;
    for (int i = 0; i < s.n_atoms; ++i)
      for (int q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
        int j = P->h_col[q];
        int bi = s.bsize[i], bj = s.bsize[j];
        for (int a = 0; a < bi; ++a)
          for (int b = 0; b < bj; ++b) {
            size_t e = (size_t)q * B * B + a * B + b;
            vals[2 * o] = cplx ? buf[2 * e] : buf[e];
            vals[2 * o + 1] = cplx ? buf[2 * e + 1] : 0.0;
            ++o;
          }
      }
    return RT_OK;
  });
}

rt_status rt_unitarity(rt_ctx* c, int32_t sys, int32_t metric_S, double* maxabs, double* meanabs) {
  return guarded(c, [&] {
    check_sys(c, sys);
    RT_REQUIRE(maxabs && meanabs, RT_EINVAL, "NULL output");
    Sys& s = *c->sys[sys];
    unitarity(c, s, metric_S ? 1 : 0, maxabs, meanabs);
    return RT_OK;
  });
}

rt_status rt_step_work(rt_ctx* c, double* flops, double* bytes) {
  return guarded(c, [&] {
    RT_REQUIRE(flops && bytes, RT_EINVAL, "NULL output");
    c->counting = true;
    c->count_flops = c->count_bytes = 0.0;
    try {
      enqueue_step(c);
    } catch (...) {
      c->counting = false;
      throw;
    }
    c->counting = false;
    *flops = c->count_flops;
    *bytes = c->count_bytes;
    return RT_OK;
  });
}

rt_status rt_step_kernels(rt_ctx* c, int64_t* kernels) {
  return guarded(c, [&] {
    RT_REQUIRE(kernels, RT_EINVAL, "NULL output");
    c->counting = true;
    c->count_flops = c->count_bytes = 0.0;
    c->count_kernels = 0;
    try {
      enqueue_step(c);
    } catch (...) {
      c->counting = false;
      throw;
    }
    c->counting = false;
    *kernels = c->count_kernels;
    return RT_OK;
  });
}

rt_status rt_profile(rt_ctx* c, int32_t enable) {
  return guarded(c, [&] {
    c->profiling = enable != 0;
    for (auto& pr : c->prof) pr = rt_ctx::Prof{};
    return RT_OK;
  });
}

rt_status rt_profile_read(rt_ctx* c, int32_t max, int32_t* n_classes, int64_t* launches, double* ms, double* flops,
                          double* bytes, char* names) {
  return guarded(c, [&] {
    RT_REQUIRE(n_classes && launches && ms && flops && bytes && names, RT_EINVAL, "NULL output");
    collect_profile(c);
    int n = std::min<int>(max, PC_N);
    for (int i = 0; i < n; ++i) {
      launches[i] = c->prof[i].launches;
      ms[i] = c->prof[i].ms;
      flops[i] = c->prof[i].flops;
      bytes[i] = c->prof[i].bytes;
      std::snprintf(names + 32 * i, 32, "%s", kProfNames[i]);
    }
    *n_classes = n;
    return RT_OK;
  });
}

struct StateHeader {
  uint64_t magic;
  int64_t host_step;
  double t_host;
  int64_t n_slots;
};

rt_status rt_get_state(rt_ctx* c, void* buf, size_t* bytes) {
  return guarded(c, [&] {
    RT_REQUIRE(bytes, RT_EINVAL, "NULL size");
    size_t need = sizeof(StateHeader) + sizeof(DevState) + sizeof(int64_t) * c->n_slots;
    for (auto& sp : c->sys) {
      Sys& s = *sp;
      need += sizeof(double2) * nvals(s, s.pK) * s.K.size();
      need += sizeof(double2) * nvals(s, s.pU);
      if (s.X) need += sizeof(double2) * nvals(s, s.pU);
    }
    if (!buf) {
      *bytes = need;
      return RT_OK;
    }
    RT_REQUIRE(*bytes >= need, RT_EINVAL, "state buffer too small");
    for (auto& sp : c->sys) {  // the state holds K and U themselves
      materialize(c, *sp, true);
      refresh_u64(c, *sp);
    }
    for (auto& sp : c->sys) {
      // and U itself: where only U - I is current (FP32 EM, ETRS, M4), U = I + (U - I)
      Sys& s = *sp;
      if (s.duf_current) launch_u_from_delta(s.dUf, s.U, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws);
    }
    char* o = (char*)buf;
    StateHeader h{0x52544b53544154ull, c->host_step, c->t_host, c->n_slots};
    memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    RT_CUDA_CHECK(cudaMemcpyAsync(o, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->ws));
    o += sizeof(DevState);
    memcpy(o, c->read_upto.data(), sizeof(int64_t) * c->n_slots);
    o += sizeof(int64_t) * c->n_slots;
    for (auto& sp : c->sys) {
      Sys& s = *sp;
      for (double2* K : s.K) {
        size_t nb = sizeof(double2) * nvals(s, s.pK);
        RT_CUDA_CHECK(cudaMemcpyAsync(o, K, nb, cudaMemcpyDeviceToHost, c->ws));
        o += nb;
      }
      size_t nu = sizeof(double2) * nvals(s, s.pU);
      RT_CUDA_CHECK(cudaMemcpyAsync(o, s.U, nu, cudaMemcpyDeviceToHost, c->ws));
      o += nu;
      if (s.X) {
        RT_CUDA_CHECK(cudaMemcpyAsync(o, s.X, nu, cudaMemcpyDeviceToHost, c->ws));
        o += nu;
      }
    }
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    *bytes = need;
    return RT_OK;
  });
}

rt_status rt_set_state(rt_ctx* c, const void* buf, size_t bytes) {
  if (!c) return RT_EINVAL;
  // validate the checkpoint before anything else: a rejected restore leaves a
  // poisoned context poisoned (its K and U may hold a partial step)
  if (c->unrecoverable) {
    c->err = "a bounded wait and its drain both gave up: copies may have landed late; the context cannot be restored";
    return RT_ESTATE;
  }
  size_t need = sizeof(StateHeader) + sizeof(DevState) + sizeof(int64_t) * c->n_slots;
  for (auto& sp : c->sys) {
    Sys& s = *sp;
    need += sizeof(double2) * nvals(s, s.pK) * s.K.size() + sizeof(double2) * nvals(s, s.pU);
    if (s.X) need += sizeof(double2) * nvals(s, s.pU);
  }
  if (!buf) {
    c->err = "NULL state";
    return RT_EINVAL;
  }
  if (bytes != need) {
    c->err = "state size does not match this context";
    return RT_EINVAL;
  }
  StateHeader h;
  memcpy(&h, buf, sizeof(h));
  if (h.magic != 0x52544b53544154ull || h.n_slots != c->n_slots) {
    c->err = "not a state of this context";
    return RT_EINVAL;
  }
  const bool was_poisoned = c->poisoned;
  c->poisoned = false;
  rt_status st = guarded(c, [&] {
    const char* o = (const char*)buf + sizeof(h);
    RT_CUDA_CHECK(cudaMemcpyAsync(c->dstate, o, sizeof(DevState), cudaMemcpyHostToDevice, c->ws));
    o += sizeof(DevState);
    memcpy(c->read_upto.data(), o, sizeof(int64_t) * c->n_slots);
    o += sizeof(int64_t) * c->n_slots;
    for (auto& sp : c->sys) {
      Sys& s = *sp;
      std::fill(s.dk_fresh.begin(), s.dk_fresh.end(), 0);  // K restored; the reference is kept
      if (!c->p.full_step) s.r_ready = false;                  // a constant U's R follows the restored U
      for (double2* K : s.K) {
        size_t nb = sizeof(double2) * nvals(s, s.pK);
        RT_CUDA_CHECK(cudaMemcpyAsync(K, o, nb, cudaMemcpyHostToDevice, c->ws));
        o += nb;
      }
      size_t nu = sizeof(double2) * nvals(s, s.pU);
      RT_CUDA_CHECK(cudaMemcpyAsync(s.U, o, nu, cudaMemcpyHostToDevice, c->ws));
      o += nu;
      if (s.X) {
        RT_CUDA_CHECK(cudaMemcpyAsync(s.X, o, nu, cudaMemcpyHostToDevice, c->ws));
        o += nu;
      }
      if (c->p.precision == RT_FP32 && s.dUf) {
        launch_u_minus_i_f32(s.U, s.dUf, s.pU->nnzb, s.pU->rowidx, s.pU->col, s.B, c->ws);
        if (s.dUH) launch_dagger32(s.dUf, s.dUH, s.pU->nnzb, s.B, c->ws);
      }
      s.u64_stale = false;  // the restored U is the FP64 propagator (the reference split rounds it per step)
    }
    c->host_step = h.host_step;
    c->t_host = h.t_host;
    RT_CUDA_CHECK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->ws));  // the restored state is sound again
    c->graph_dirty = true;
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    return RT_OK;
  });
  if (st != RT_OK && was_poisoned) c->poisoned = true;  // a failed restore clears nothing
  return st;
}

rt_status rt_debug_check(rt_ctx* c, int64_t* n_checked) {
  return guarded(c, [&] {
    int64_t n = 0;
    for (size_t si = 0; si < c->sys.size(); ++si) {
      Sys& s = *c->sys[si];
      for (auto& kv : s.tcache) {
        const TripleKey& key = kv.first;
        const Triples& T = kv.second->t;
        std::vector<int32_t> items((size_t)T.n_items);
        std::vector<int64_t> ptr((size_t)T.n_items + 1, 0);
        std::vector<int32_t> ab((size_t)(2 * T.n_triples));
        if (T.n_items) {
          RT_CUDA_CHECK(cudaMemcpyAsync(items.data(), T.item_blk, sizeof(int32_t) * items.size(),
                                        cudaMemcpyDeviceToHost, c->ws));
          RT_CUDA_CHECK(cudaMemcpyAsync(ptr.data(), T.ptr, sizeof(int64_t) * ptr.size(), cudaMemcpyDeviceToHost, c->ws));
        }
        if (T.n_triples)
          RT_CUDA_CHECK(cudaMemcpyAsync(ab.data(), T.ab, sizeof(int2) * (size_t)T.n_triples, cudaMemcpyDeviceToHost,
                                        c->ws));
        RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
        int64_t bad = -1;
        std::string why;
        const bool ok = check_triples_host(
            s.n_atoms, key.A->h_rowptr.data(), key.A->h_col.data(), key.ad, key.B->h_rowptr.data(),
            key.B->h_col.data(), key.bd, key.C->h_rowptr.data(), key.C->h_col.data(), key.up, T.n_items, items.data(),
            ptr.data(), ab.data(), T.n_triples, &bad, &why);
        RT_REQUIRE(ok, RT_EINTERNAL,
                   "triple list of system " + std::to_string(si) + " (P_A r = " + std::to_string(key.A->radius) +
                       (key.ad ? " dagger" : "") + ", P_B r = " + std::to_string(key.B->radius) +
                       (key.bd ? " dagger" : "") + ", P_C r = " + std::to_string(key.C->radius) +
                       (key.up ? " upper" : "") + ") fails at item " + std::to_string(bad) + ": " + why);
        ++n;
      }
    }
    if (n_checked) *n_checked = n;
    return RT_OK;
  });
}

rt_status rt_debug_inject(rt_ctx* c, uint32_t flags) {
  return guarded(c, [&] {
    const uint32_t known = RT_FAULT_HOTELLING_MAXITER1 | RT_FAULT_NAN_IN_H | RT_FAULT_WAIT_TIMEOUT_0;
    RT_REQUIRE((flags & ~known) == 0, RT_EINVAL, "unknown fault flags");
    if (flags & RT_FAULT_NAN_IN_H) {
      Sys& s = *c->sys[0];
      const double nan = std::numeric_limits<double>::quiet_NaN();
      RT_CUDA_CHECK(cudaMemcpyAsync(s.H0, &nan, sizeof(double), cudaMemcpyHostToDevice, c->ws));
      if (s.T0) RT_CUDA_CHECK(cudaMemcpyAsync(s.T0, &nan, sizeof(double), cudaMemcpyHostToDevice, c->ws));
      if (!s.V.empty()) RT_CUDA_CHECK(cudaMemcpyAsync(s.V[0], &nan, sizeof(double), cudaMemcpyHostToDevice, c->ws));
      RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    }
    c->inject |= flags & (RT_FAULT_HOTELLING_MAXITER1 | RT_FAULT_WAIT_TIMEOUT_0);
    return RT_OK;
  });
}

rt_status rt_synchronize(rt_ctx* c) {
  return guarded(c, [&] {
    RT_CUDA_CHECK(cudaStreamSynchronize(c->ws));
    check_device_error(c);
    return RT_OK;
  });
}

const char* rt_last_error(rt_ctx* c) {
  if (!c) return "NULL context";
  return c->err.c_str();
}

void rt_destroy(rt_ctx* c) {
  if (!c) return;
  if (c->ws) cudaStreamSynchronize(c->ws);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (auto& pe : c->pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto& e : c->ev_free) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  c->arena.release_all();
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ws) cudaStreamDestroy(c->ws);
  delete c;
}

}  // extern "C"
