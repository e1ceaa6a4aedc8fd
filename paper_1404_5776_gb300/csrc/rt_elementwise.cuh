// Declarations of the elementwise / reduction launches (elementwise.cu).
#pragma once

#include "rt_internal.cuh"

namespace rt {

struct FieldParams {
  int kind = RT_FIELD_NONE;
  int dir = 0;
  double E0 = 0.0, t0 = 0.0, sigma = 1.0, omega = 0.0;
};

// Device-resident step state (read by kernels so that a captured step graph
// can be replayed without new kernel arguments).
constexpr int RT_MAX_SLOTS = 256;  // (system, kick) pairs
struct DevState {
  int64_t step;
  double t;
  double E[5];  // field at t + dt/2, t, t + dt, t1, t2 (Gauss-Legendre points of M4)
  double hot_resid;
  int hot_iters;
  int pad;
  unsigned long long herm_bits[RT_MAX_SLOTS];
};

void launch_begin_step(DevState* s, const FieldParams& f, double dt, int n_herm, cudaStream_t st);
void launch_end_step(DevState* s, double dt, cudaStream_t st);
// Hm = H0 - s->E[which] * D (s == nullptr: Hm = H0 - scale * D)
void launch_field_axpy(const double* H0, const double* D, const DevState* s, int which, double scale, double* Hm,
                       int64_t n, cudaStream_t st);
// M4 exponent on P_U: Om = -i dt/2 (T1 + T2) - (sqrt(3) dt^2 / 12) (C21 - C12)
void launch_m4_omega(const double* T1, const double* T2, const int32_t* u_to_t, const double* C21, const double* C12,
                     double dt, double2* Om, int64_t nnzb_u, int B, cudaStream_t st);
void launch_taylor_init(void* U, bool fp32, int64_t nnzb_u, const int32_t* u_rowidx, const int32_t* u_col,
                        const void* T, bool t_fp32, const int32_t* u_to_t, int B, double c1, int c1_imag, int ident,
                        cudaStream_t st);
void launch_identity(double* X, bool cplx, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B,
                     double scale, cudaStream_t st);
void launch_restrict(const double* src, double* dst, const int32_t* map, int64_t nnzb_dst, int B, int mode,
                     cudaStream_t st);
void launch_cn_operands(const double* S, const int32_t* a_to_s, const double* H, const int32_t* a_to_h, double c,
                        double2* A, double2* Bm, int64_t nnzb_a, int B, cudaStream_t st);
int reduce_blocks(int64_t n);
void launch_sum(const double* v, int64_t n, double* part, double sqrt_div, double* out, double* out2,
                cudaStream_t st);
void launch_traces(const double2* K, int64_t nnzb, const int32_t* rowidx, const int32_t* col, const int32_t* bsize,
                   int B, const double* S, const int32_t* ks_map, const double* Dx, const double* Dy,
                   const double* Dz, const int32_t* kd_map, double* part, const DevState* st, int herm_slot,
                   double* ring, int capacity, int n_slots, int slot_index, cudaStream_t s,
                   const double* ref = nullptr, double* out = nullptr);
// Arguments of the traces of one (system, kick) pair (as launch_traces takes them)
struct TracePair {
  const double2* K;
  int64_t nnzb;
  const int32_t *rowidx, *col, *bsize;
  int B;
  const double* S;
  const int32_t* ks_map;
  const double *Dx, *Dy, *Dz;
  const int32_t* kd_map;
  int herm_slot, slot_index;
  const double* ref;
};
// launch_traces for every pair of a device table in two launches: nb CTAs per pair (reduce_blocks of the
// largest pair), partials in part[n_pairs][nb][8], one observables record per pair
void launch_traces_grouped(const TracePair* tab, int n_pairs, int nb, double* part, const DevState* st, double* ring,
                           int capacity, int n_slots, cudaStream_t s);
// dU = U - I stochastically rounded to FP32 (draws keyed on s->step and the element) and its per-block
// conjugate transpose dUH (if non-null), from an FP64 U; with `planar` (13-function blocks) dU is written
// column-planar (per column: real parts of rows 0..15, then imaginary parts), dUH in the row layout
void launch_round_u_sr(const double2* U, float2* dU, float2* dUH, int64_t nnzb, const int32_t* rowidx,
                       const int32_t* col, int B, const DevState* s, cudaStream_t st, bool planar = false);
void launch_zaxpy(double2* z, const double2* x, const double2* y, double a, int64_t n, cudaStream_t st);
void launch_axpy32(float2* z, const float2* x, const float2* y, float a, int64_t n, cudaStream_t st);
void launch_m4_omega32(const double* T1, const double* T2, const int32_t* u_to_t, const float* C21, const float* C12,
                       double dt, float2* Om, float2* dU, bool first_term, int64_t nnzb_u, int B, cudaStream_t st);
// V[q] += coef * Q[map[q]] (real Q into the real or, with imag, the imaginary part of V; map null = same
// blocks, -1 = no block)
void launch_acc_real(double2* V, const double* Q, const int32_t* map, int64_t nnzb_v, int B, double coef, int imag,
                     cudaStream_t st);
constexpr int RT_MAX_POLY = 32;
struct PolyTerms {
  const double2* v[RT_MAX_POLY];
};
// FP32 copies of V_1..V_deg (v[0] unused) for the FP32 tail of the Horner pass
struct PolyTerms32 {
  const float2* v[RT_MAX_POLY];
};
// b = (float)a for n complex values (dense, same element order)
void launch_z2c(const double2* a, float2* b, int64_t n, cudaStream_t st);
// U = sum_{m<=deg} E^m V_m at E = s->E[which] (Horner, FP64); writes U (FP64, if non-null) and/or
// dU = U - I with its per-block conjugate transpose dUH in FP32 (padded rows), if non-null, rounded to
// nearest or, with `stochastic`, stochastically (draws keyed on s->step and the element); with `planar`
// (13-function blocks) dU is written column-planar as in launch_round_u_sr
// tail (with dU only, stochastic): U = V_0 + E q(E), q(E) = sum_{m>=1} E^(m-1) V_m by Horner in FP32 over
// tail->v[1..deg] and V_0 + E q in FP64 (two FP64 FMAs per element instead of 2 deg); q's FP32 rounding
// is far below the stochastic rounding of dU that follows
void launch_field_poly(const PolyTerms& V, int deg, const DevState* s, int which, double2* U, float2* dU,
                       float2* dUH, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B, cudaStream_t st,
                       bool stochastic = false, bool planar = false, const PolyTerms32* tail = nullptr);
// R = sum_{p<=deg} E^p C_p at E = s->E[which] (Horner, FP64) on the upper blocks of a pattern
void launch_poly_upper(const PolyTerms& C, int deg, const DevState* s, int which, double2* R, int64_t nnzb,
                       const int32_t* rowidx, const int32_t* col, int B, cudaStream_t st);
int launch_unitarity_dev(const double2* E, int64_t nnzb, const int32_t* rowidx, const int32_t* col,
                         const int32_t* bsize, int B, const double* S, const int32_t* us_map, double* part_max,
                         double* part_sum, cudaStream_t st);
void launch_inf_norm(const double* S, const int32_t* rowptr, const int32_t* col, const int32_t* bsize, int B,
                     int n_atoms, double* rows_tmp, double* out, cudaStream_t st);
void launch_cheb_step(const double* TY, const double* Y, const double* Yp, double* Yn, double* Kacc, double a,
                      double w, double c, int first, int64_t n, cudaStream_t st);
void launch_scale(double* v, double c, int64_t n, cudaStream_t st);
void launch_symmetrise_to_complex(const double* Kr, double2* K, int64_t nnzb, const int32_t* rowidx,
                                  const int32_t* col, const int32_t* tmap, const int32_t* bsize, int B,
                                  cudaStream_t st);
void launch_d2f_pad(const double* a, float* b, int64_t nnzb, int B, bool cplx, cudaStream_t st);
void launch_dagger32(const float2* dU, float2* dUH, int64_t nnzb, int B, cudaStream_t st);
// Y <- 2I - Y (FP32 complex, FP32 block layout, in place; identity on diagonal blocks)
void launch_two_i_minus32(float2* Y, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B,
                          cudaStream_t st);
// FP32 complex (FP32 block layout) -> FP64 complex dense blocks
void launch_f2d_unpad(const float2* a, double2* b, int64_t nnzb, int B, cudaStream_t st);
void launch_delta_w(const double2* K, const int32_t* m_to_k, const float2* Mf, float2* Wf, int64_t nnzb_m, int B,
                    cudaStream_t st);
void launch_set_hot(DevState* s, const double* resid, int iters, cudaStream_t st);
void launch_u_from_delta(const float2* dU, double2* U, int64_t nnzb, const int32_t* rowidx, const int32_t* col, int B,
                         cudaStream_t st);
void launch_u_minus_i_f32(const double2* U, float2* dU, int64_t nnzb, const int32_t* rowidx, const int32_t* col,
                          int B, cudaStream_t st);

}  // namespace rt
