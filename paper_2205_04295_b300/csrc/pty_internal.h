// Internal declarations shared by the host API (pty_api.cu) and the kernel
// launchers (pty_rpie.cu, pty_refine.cu, pty_grad.cu).  Not part of the ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <complex>

namespace pty {

struct UpdArgs {
  float alpha_O, alpha_P, beta, gamma, eps, reg_eps;
};

// Launch geometry of the three passes for one (W, M).
struct Tiling {
  int W, M;
  int npl;       // far-field planes per patch in the scratch (M, or M + 2 refining)
  int xo;        // 1: passes A/B also transform the crop itself (plane M)
  int refine;    // 1: pass C also row-transforms the refined crop (plane M + 1)
  int R;         // rows per CTA, row passes
  int ppc;       // patches per CTA, row passes
  int CB;        // columns per CTA, column pass
  int ppcb;      // patches per CTA, column pass
  int ppcc;      // patches per CTA, pass C (ppc unless re-chosen for a chunk)
  int resA, resB, resC;  // CTAs of the three pass kernels resident on the device (0: unknown)
  int thrA, thrB, thrC;
  size_t smA, smB, smC, smI;  // dynamic shared memory (bytes)
  size_t smA_staged;          // pass A with its probe rows in shared memory (batched form)
  int n_pmax;    // CTAs of the probe-apply kernel (= partial maxima)
  int pstage;    // 1: pass C copies its probe rows to shared memory (when that
                 // costs it no CTA per SM), 0: reads them through L1 at use
};

bool supported_W(int W);
// The pass kernels' launch bounds (rows 256, columns 384 threads) and the
// opt-in shared memory hold for this tiling.
bool tiling_fits(const Tiling& t);

// Largest dynamic shared memory a block may opt in to on the current device.
// Every kernel's opt-in limit is set to this value: the attribute is global
// per kernel function, so a limit sized for one tiling would reject another.
int smem_optin();
// Shared memory per SM (bytes).
int smem_per_sm();
// Let `func` use all dynamic shared memory the device allows beside its own
// static shared memory.
cudaError_t allow_max_smem(const void* func);

// Record a failure message for pty_last_error() on this thread; returns code.
int set_error(int code, const char* fmt, ...);
// R_req / ppc_req / CB_req > 0 override the defaults (callers validate them).
Tiling make_tiling(int W, int M, bool refine = false, int max_threads_b = 512, int R_req = 0,
                   int ppc_req = 0, int CB_req = 0);
int lanes_per_line(int W);
cudaError_t set_smem_limits(const Tiling& t);
// Fill t.resA / resB / resC (after set_smem_limits).
void fill_residency(Tiling& t);
// The tiling for a chunk of n patches: the patches per CTA of pass A (ppc)
// and of the column pass (ppcb) re-chosen near the tuned values so that each
// kernel's CTAs end close to a whole number of waves (pass A's dynamic shared
// memory follows ppc).  Neither changes a result (no sum runs across a CTA's
// patches there); pass C keeps ppcc, whose probe-sum slots the results do
// depend on.
Tiling tiling_for_chunk(const Tiling& t, int n);

// Twiddle table of the line FFTs: slot e holds w_W^m = exp(-2 pi i m / W) with
// m = tw_exponent(W, e) (host, double -> float).
void make_twiddles(int W, float2* out);

// ---- the three passes of one chunk of a group -----------------------------
cudaError_t launch_rows_fwd(const Tiling& t, const float2* O, int Hx,
                            const float2* P, const int* ids, const int2* corners,
                            int npatch, const float2* tw, float2* scratch,
                            float* omax_part, cudaStream_t s);
cudaError_t launch_rows_fwd_plain(const Tiling& t, const float2* O, int Hx,
                                  const float2* P, const int* ids, const int2* corners,
                                  int npatch, const float2* tw, float2* scratch,
                                  float* omax_part, cudaStream_t s);
// tm (may be NULL): tensor map of the scratch for TMA staging (see
// encode_far_field_map); a TMA wait that times out sets *err.  xb >= 0
// (XCORR_B): also write the model intensity and the counts into scratch
// planes xb, xb + 1.  plane0: the plane of the tensor map at which `scratch`
// starts (a chunk placed further into the scratch).
cudaError_t launch_cols(const Tiling& t, float2* scratch, const uint16_t* I,
                        const int* ids, int npatch, const float2* tw, float inv_w,
                        float eps, float* err_part, const CUtensorMap* tm, int* err,
                        cudaStream_t s, int xb = -1, int plane0 = 0);
// Fourier-domain step of the gradient (amplitude loss, delta-smoothed).
cudaError_t launch_cols_grad(const Tiling& t, float2* scratch, const uint16_t* I,
                             const int* ids, int npatch, const float2* tw, float inv_w,
                             float delta, float* loss_part, int npl, const CUtensorMap* tm,
                             int* err, cudaStream_t s);
// Tensor map over `planes` W x W complex64 planes at `base`, box CB x W x 1
// (the column pass's block of one plane).  False if the driver entry point
// is missing or the arguments break the TMA rules (the caller then stages
// with cp.async).
bool encode_far_field_map(const void* base, int W, size_t planes, int CB, CUtensorMap* out);
// ---- differentiable forward model and adjoint (pty_grad.cu) ---------------
cudaError_t launch_grad_rows_fwd(const Tiling& t, const float2* O, int Hx, const float2* P,
                                 const int* ids, const float* pos, int npatch,
                                 const float2* tw, float2* scratch, int npl, cudaStream_t s);
cudaError_t launch_grad_rows_inv(const Tiling& t, const float2* O, int Hx, const float2* P,
                                 const int* ids, const float* pos, int npatch,
                                 float2* scratch, int npl, const float2* tw, float2* gP_part,
                                 int accumulate, float* gpos_part, cudaStream_t s);
cudaError_t launch_grad_scatter(int W, int M, float2* gO, int Hx, const int* ids,
                                const float* pos, int npatch, const float2* scratch, int npl,
                                cudaStream_t s);
cudaError_t launch_grad_finish(const Tiling& t, int nslots, const float2* gP_part, float2* gP,
                               const float* gpos_part, int N, float* gpos,
                               const float* loss_part, size_t nloss, float* loss,
                               double* tmp, cudaStream_t s);
cudaError_t set_grad_smem(const Tiling& t);

cudaError_t launch_rows_inv(const Tiling& t, float2* O, int Hx, const float2* P,
                            const int* ids, const int2* corners, int npatch,
                            float2* scratch, const float* omax_part,
                            const float* pmax_part, const float2* tw,
                            const UpdArgs& a, float2* pnum, float* pden,
                            float* osum, int accumulate, int* err, cudaStream_t s,
                            int refine = -1);  // -1: t.refine; 0: no o'_j row DFTs
cudaError_t launch_probe_apply(const Tiling& t, float2* P, const float2* pnum,
                               const float* pden, const float* osum, int nslots,
                               float alpha_P, float reg_eps, float* pmax_part,
                               cudaStream_t s);
cudaError_t launch_pmax(const Tiling& t, const float2* P, float* pmax_part,
                        cudaStream_t s);
// Probe-mode orthogonalisation (pty_modes.cu): Gram matrix (M*M double2,
// row k column l = sum_r conj(P_k) P_l), the host Hermitian eigensolver
// (decreasing eigenvalues; 0 on success) and the in-place mixing
// P'_m = sum_k V[k][m] P_k.
cudaError_t launch_gram(const float2* P, int M, int WW, void* G, cudaStream_t s);
int hermitian_eig(int M, const std::complex<double>* A, double* w, std::complex<double>* V);
cudaError_t launch_mix(float2* P, int M, int WW, const float2* V, cudaStream_t s);

// Error normalised by 1/sum(I): inv_sumI, or the device sum when sum_dev != NULL.
// tmp: kErrPartsMax doubles of device scratch.
constexpr int kErrPartsMax = 296;
cudaError_t launch_err_reduce(const float* err_part, size_t n, double inv_sumI,
                              const unsigned long long* sum_dev, float* out, double* tmp,
                              cudaStream_t s);
cudaError_t launch_cols_intensity(const Tiling& t, const float2* scratch,
                                  const int* ids, int npatch, const float2* tw,
                                  float inv_w, float* out, cudaStream_t s);
// ---- XCORR_A / XCORR_B registration and the Adam step (pty_refine.cu) ------
struct RefGeo {
  int W, U, K;   // fine grid K = ceil(1.5 U) points per axis
  int CBX, RX;   // columns / rows per CTA of the correlation passes
  int RB;        // rows of X per CTA of the upsampled matrix DFT
  size_t smX, smR, smU;
  bool tc;       // fine-grid DFT on the tensor cores (K <= 32 and not turned off)
};
// tc: take the tensor-core form of the fine-grid DFT where it applies (K <= 32)
RefGeo make_refgeo(int W, int U, bool tc = true);
cudaError_t set_refine_smem(const RefGeo& g);
// roots exp(+2 pi i n / (U W)), n = 0..U W - 1 (host, double -> float)
void make_up_roots(int W, int U, float2* out);
// Forward row DFTs, in place, of planes plane .. plane + nplanes - 1 of every
// patch: XCORR_B's model intensity and counts (planes M, M + 1), XCORR_A's
// refined crop (plane M + 1) as the three-pass path leaves it.
cudaError_t launch_xcorrb_rows(const RefGeo& g, float2* scratch, int npl, int plane,
                               int nplanes, int npatch, const float2* tw, cudaStream_t s);
cudaError_t launch_xcorr_cols(const RefGeo& g, float2* scratch, int npl, int M, int npatch,
                              const float2* tw, cudaStream_t s);
cudaError_t launch_xcorr_rows(const RefGeo& g, const float2* scratch, int npl, int M,
                              int npatch, const float2* tw, float* cval, int* cidx,
                              cudaStream_t s);
// part: npatch * (W / 16) * K * K complex partial sums of the fine grid;
// done: npatch zeroed counters (the tensor-core form's last-CTA detection,
// left at zero); err: status word set by a tensor-core wait that gave up
cudaError_t launch_updft(const RefGeo& g, float2* scratch, int npl, int M, const int* ids,
                         int npatch, const float* cval, const int* cidx, const float2* roots,
                         float2* part, float* shift, float* gap, int* done, int* err,
                         cudaStream_t s);
cudaError_t launch_adam(float* pos, float* m, float* v, const float* g, int N, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, float max_step,
                        float ymax, float xmax, cudaStream_t s);

// ---- batched persistent form (pty_batch.cu) --------------------------------
struct BatchProb {
  int W, M, N, Hx, R, ppc, CB, n_pmax;
  float inv_w;
  int update_probe;
  UpdArgs a;
  double inv_sumI;
  const float2* tw;
  float2* O;
  float2* P;
  const uint16_t* I;
  const int2* corners;
  const int* gpos;
  float2* scratch;
  float2* pnum;
  float* pden;
  float* osum;
  float* omax_part;
  float* err_part;
  float* pmax_part;
  float* err_iter;
  size_t err_part_n;
};
enum { BT_ROWS = 0, BT_COLS = 1, BT_ROWS_INV = 2, BT_PROBE = 3, BT_ERR = 4 };
struct BatchTask {
  int prob, kind, x0, x1;   // problem, pass, tile range [x0, x1)
  int y, ids_off, npatch, flag;  // patch sub-block, chunk offset in the group list, chunk size,
                                 // accumulate (rows_inv) or slot count (probe)
  unsigned need;            // tasks of this problem that must be complete first
  int it, pad0, pad1;
};
size_t batch_smem(const Tiling& t);
// Largest co-resident grid for `smem` bytes of dynamic shared memory.
cudaError_t batch_grid(size_t smem, int* ctas);
cudaError_t launch_batch(const BatchProb* probs, const BatchTask* tasks, int ntask,
                         unsigned* next, unsigned* done, int* error,
                         unsigned long long timeout_ns, int ctas, size_t smem,
                         cudaStream_t s);

// ---- fused single-kernel patch path for W <= 128 (pty_patch.cu) ----------
// One cluster of S CTAs per patch: CTA s holds rows [s W/S, (s+1) W/S) of
// every mode's W x W plane and, between two transposes through distributed
// shared memory, columns [s W/S, (s+1) W/S); the 2-D DFTs, the modulus
// constraint and the object / probe-sum updates run there.  The far-field
// scratch is written only for the registration's crop planes.
struct PatchGeo {
  int W, M, S;     // S CTAs per patch (1, 2, 4, 8; W / S a multiple of 8)
  int NL, NT;      // lines per round and threads per CTA
  size_t sm;       // dynamic shared memory (bytes)
  int ncap;        // clusters resident at once (0: the launch cannot run)
};
struct PatchArgs {
  float2* O;
  int Hx, M;
  const float2* P;
  const uint16_t* I;
  const int* ids;
  const int2* corners;
  int npatch, NL;
  const float2* tw;
  float inv_w;
  UpdArgs a;
  const float* pmax_part;
  int n_pmax;
  float2* pnum;
  float* pden;
  float* osum;
  int accumulate;   // add to the probe sums of the slots (a later chunk)
  float* err_part;
  int nb;           // error partial slots per pattern (the first gets the sum)
  float2* scratch;
  int npl;
  int refine;       // 0; 1: XCORR_A crop planes M, M + 1; 2: XCORR_B planes M, M + 1
};
// S = 0 or an unsupported (W, M, S): ncap = 0.  Queries the device.
PatchGeo make_patch_geo(int W, int M, int S);
cudaError_t set_patch_smem(int W);
// nclusters <= ncap clusters over a.npatch patches; slot c = cluster c.
cudaError_t launch_patch(const PatchGeo& g, const PatchArgs& a, int nclusters, cudaStream_t s);

cudaError_t launch_fft2(void* data, int W, int batch, int inverse,
                        const float2* tw, cudaStream_t s);
cudaError_t launch_finite_check(const float* p, size_t n, int* flag,
                                cudaStream_t s);

}  // namespace pty
