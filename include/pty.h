/*
 * pty.h -- C ABI of libpty, a B300 (sm_103a) implementation of mixed-state
 * rPIE ("M-rPIE") ptychographic reconstruction with Adam-controlled XCORR_A
 * position refinement, after Guzzi et al., "A modular software framework for
 * the design and implementation of ptychography algorithms"
 * (arXiv 2205.04295).
 *
 * Conventions shared by every call:
 *   - Every function returns PTY_OK (0) or a PTY_E* code; on failure
 *     pty_last_error() returns a message for the calling thread.  No C++
 *     exception crosses this boundary.
 *   - Complex arrays are interleaved complex64 (float re, float im), row-major.
 *   - Object O: Hy x Hx.  Probe P: M modes of W x W ("P_p" of Eq. 4).
 *   - Diffraction stack I: N patterns of W x W uint16 photon counts, stored
 *     detector-centred (zero spatial frequency at pixel (W/2, W/2)).
 *   - Positions: N pairs (y, x), float32, the top-left corner of the crop box
 *     o_j in object pixels.  rPIE crops at floor(pos + 0.5); the
 *     differentiable form samples bilinearly at the exact position.
 *   - mem_kind PTY_MEM_HOST: a host pointer (pageable or pinned);
 *     PTY_MEM_DEVICE: a device pointer on the handle's current device.
 *   - Work is ordered on the handle's stream.  Calls that return host data
 *     synchronise that stream; all others may return before the GPU is done.
 *   - Pattern sizes supported by the kernels: W in {32, 64, 96, 128, 192, 256}.
 *   - A handle is not thread-safe: one thread at a time per handle.
 */
#ifndef PTY_H_
#define PTY_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTY_ABI_VERSION 3

enum {
  PTY_OK = 0,
  PTY_EINVAL = 1,   /* bad argument: null pointer, size, unsupported W, ... */
  PTY_ENOMEM = 2,   /* device allocation (or the caller's allocator) failed */
  PTY_ECUDA = 3,    /* a CUDA runtime call failed */
  PTY_EDATA = 4,    /* data outside the model: crop outside O, non-finite values */
  PTY_ETIMEOUT = 5, /* a bounded device-side wait gave up */
  PTY_ESTATE = 6    /* call out of order, e.g. iterations before pty_set_data */
};

enum { PTY_MEM_HOST = 0, PTY_MEM_DEVICE = 1 };

typedef struct pty_handle pty_handle;

/* Optional device allocator: return a device pointer of at least `bytes`
 * bytes usable on `stream`, or NULL on failure.  `free` releases it. */
typedef void* (*pty_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pty_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
  int W;                /* pattern side length (pixels) */
  int M;                /* number of probe modes, >= 1 */
  int N;                /* number of scan positions, >= 1 */
  int Hy, Hx;           /* object size, >= W */
  void* stream;         /* cudaStream_t; NULL = the legacy default stream */
  pty_alloc_fn alloc;   /* NULL = cudaMalloc / cudaFree */
  pty_free_fn free;
  void* alloc_ctx;
  size_t scratch_bytes; /* cap on the far-field scratch; 0 = 64 MiB.  The
                           scratch holds M far-field waves per patch of a chunk
                           of one group; a smaller cap means smaller chunks. */
  int flags;            /* PTY_FLAG_* bits, 0 = defaults */
} pty_problem_desc;

/* Take the registration's fine-grid matrix DFT on the FP32 cores instead of
 * the tensor cores (3xTF32 tcgen05 MMAs, the default wherever K <= 32). */
#define PTY_FLAG_FP32_REGISTRATION 1

/* Update parameters of M-rPIE (M-rPIE section, Eqs. 5-7). */
typedef struct {
  float alpha_O;   /* object step size alpha_O (Eq. 6) */
  float alpha_P;   /* probe step size alpha_P (Eq. 5) */
  float beta;      /* probe regulariser beta (Eq. 5); beta = gamma = 1 is M-ePIE */
  float gamma;     /* object regulariser gamma (Eq. 6) */
  float eps;       /* modulus-constraint guard: f = sqrt(I)/(sqrt(S)+eps), in
                      amplitude units (sqrt photons); 1 regularises pixels whose
                      model is darker than one photon */
  float reg_eps;   /* relative guard added to both update denominators; where
                      a denominator is exactly 0 the update is skipped */
  int max_group;   /* positions per disjoint group: 0 = unlimited, 1 = the
                      paper's sequential order */
  int update_probe;/* 0 = hold the probe fixed */
} pty_rpie_params;

/* Position refinement (Adam-based position refinement section,
 * Eqs. 8-9, Algorithm 1). */
typedef struct {
  int upsample;    /* U: registration resolution 1/U pixel; K = ceil(1.5 U) */
  float lr;        /* Adam step size (pixels) */
  float b1, b2;    /* Adam moment decays */
  float eps;       /* Adam denominator guard */
  int start_iter;  /* first iteration (counted over the handle's life) that refines */
  float max_step;  /* per-axis clamp of one step; 0 = none */
  int point;       /* where the error signal is taken (Fig. 2): PTY_XCORR_A (0),
                      the crop o_j against its update o'_j in the object plane;
                      PTY_XCORR_B (1), the model intensity sum_p |Psi_p|^2
                      against the measured counts I_j in the detector plane */
} pty_refine_params;

enum { PTY_XCORR_A = 0, PTY_XCORR_B = 1 };

/* Message describing the last failure on this thread ("" if none). */
const char* pty_last_error(void);
int pty_abi_version(void);

/* Create a problem; allocates all device state on the current device.
 * Ownership: the handle owns its device memory until pty_destroy. */
int pty_init_problem(const pty_problem_desc* d, pty_handle** out);
int pty_destroy(pty_handle* h);

/* Copy in the data and the initial guesses (stream-ordered; the caller keeps
 * its buffers).  I: N*W*W uint16, pos: N*2 float, O0: Hy*Hx complex64,
 * P0: M*W*W complex64, all of the same mem_kind.  Fails with PTY_EDATA if a
 * crop box leaves the object or a value is not finite.  Resets the Adam
 * state and the iteration counter. */
int pty_set_data(pty_handle* h, const uint16_t* I, const float* pos,
                 const void* O0, const void* P0, int mem_kind);

/* As pty_set_data, but a host pattern stack I is not copied here: the next
 * pty_run_iterations uploads it group by group on a second stream (one
 * cudaMemcpyAsync per run of consecutive pattern indices, one event per
 * group), so that group g waits only for its own patterns while the copies
 * of later groups overlap the passes of earlier ones.  Any other call that
 * reads the data uploads the remainder first.  The caller keeps I valid and
 * unchanged until that upload has completed on the GPU (after the run, e.g.
 * once a later call has synchronised the stream); page-locked I makes the
 * copies asynchronous.  pos, O0 and P0 are copied and checked before return.
 * With device memory it equals pty_set_data without its final synchronise.
 * No counterpart in the paper: an input pipeline for end-to-end runs. */
int pty_set_data_async(pty_handle* h, const uint16_t* I, const float* pos,
                       const void* O0, const void* P0, int mem_kind);

/* Optional scan order used by the greedy grouping: a permutation of 0..N-1
 * (host memory), or NULL for index order.  (The random draw, if any, is the
 * caller's.) */
int pty_set_scan_order(pty_handle* h, const int32_t* order);

/* n_iter M-rPIE iterations (Eqs. 4-7) over the disjoint-group schedule.
 * err_out (host, may be NULL) receives n_iter normalised errors
 * sum (sqrt S - sqrt I)^2 / sum I; requesting them synchronises. */
int pty_run_iterations(pty_handle* h, int n_iter, const pty_rpie_params* p,
                       float* err_out);

/* n_iter iterations with registration of every position and an Adam step
 * of every position at the end of each iteration (once the handle's
 * iteration count reaches r->start_iter); r->point picks XCORR_A (the crop
 * before and after its update) or XCORR_B (model against measured
 * detector-plane intensity), the two switch positions of Fig. 2.  Positions
 * are clamped to keep the crops inside O.  shift_out (host, N*2, may be
 * NULL) receives the last measured shift g_j = -argmax xcorr(a_j, b_j). */
int pty_refine_positions(pty_handle* h, int n_iter, const pty_rpie_params* p,
                         const pty_refine_params* r, float* err_out,
                         float* shift_out);

/* Relative gap between the best and the second-best fine-grid value of each
 * position's last registration, N floats: values near 0 flag near-ties whose
 * argmax FP32 and FP64 may resolve differently. */
int pty_get_refine_gaps(pty_handle* h, float* dst, int mem_kind);

/* Run only groups [g_begin, g_end) of the current grouping, without touching
 * positions or the iteration counter (for sampled checks of one full-size
 * launch sequence).  err_out (host, may be NULL): one value, the error
 * numerator over those groups divided by sum I. */
int pty_run_groups(pty_handle* h, int g_begin, int g_end,
                   const pty_rpie_params* p, float* err_out);

/* Current grouping (computed from the current positions): *n_groups, and if
 * non-NULL group_ptr (n_groups+1) and group_pos (N), host memory. */
int pty_get_groups(pty_handle* h, int* n_groups, int32_t* group_ptr,
                   int32_t* group_pos);

/* Copies out / in.  Sizes as in pty_set_data; Adam state m, v: N*2 float. */
int pty_get_object(pty_handle* h, void* dst, int mem_kind);
int pty_set_object(pty_handle* h, const void* src, int mem_kind);
int pty_get_probe(pty_handle* h, void* dst, int mem_kind);
int pty_set_probe(pty_handle* h, const void* src, int mem_kind);
int pty_get_positions(pty_handle* h, float* dst, int mem_kind);
int pty_set_positions(pty_handle* h, const float* src, int mem_kind);
int pty_get_adam_state(pty_handle* h, float* m, float* v, int* t, int* iter,
                       int mem_kind);
int pty_set_adam_state(pty_handle* h, const float* m, const float* v, int t,
                       int iter, int mem_kind);

/* Launch geometry of the plain M-rPIE passes, for tuning (0 = default):
 * R rows per CTA of the row passes (M * R * lanes <= 256 threads), ppc
 * patches per CTA of the row passes, CB columns per CTA of the column pass
 * (2, 4, 8 or 16, dividing W/2; M * CB * lanes <= 384 threads), scratch_bytes
 * the far-field chunk budget (also the chunk of the differentiable form,
 * whose per-patch passes take full chunks across its groups),
 * ppcb patches per CTA of the column pass.
 * fused = S > 0 (W <= 128 only) replaces the three passes of the M-rPIE
 * section's per-patch update (Eqs. 1, 2, 4-7) by one kernel per group: a
 * thread-block cluster of S CTAs per patch (S = 1, 2, 4 or 8, W / S a
 * multiple of 8), each CTA holding W / S rows of every mode's W x W plane in
 * shared memory and, between two transposes through distributed shared
 * memory, W / S columns, so that a patch makes one trip to global memory
 * (no far-field scratch); PTY_EINVAL where the slabs do not fit.  Registration (pty_refine_positions) runs on it too; the
 * differentiable form and the batched form keep their own kernels.  Results
 * do not depend on the tiling except through the summation order of the
 * probe sums.  The project's autotuner (paper_2205_04295_b300/autotune.py)
 * searches these. */
typedef struct {
  int R, ppc, CB;
  size_t scratch_bytes;
  int ppcb;         /* patches per CTA of the column pass (0 = default) */
  int fused;        /* slabs per mode of the fused patch kernel (0 = three passes) */
} pty_tiling;
int pty_set_tiling(pty_handle* h, const pty_tiling* t);
int pty_get_tiling(pty_handle* h, pty_tiling* t);

/* Launch accounting, for benchmarks.  mode 0: count launches only (always
 * on); 1: also time every kernel launch with CUDA events recorded on the
 * handle's stream.  pty_get_stats synchronises the stream, fills *out with
 * the totals since the last reset and, if reset != 0, zeroes them. */
enum { PTY_K_ROWS_FWD = 0, PTY_K_COLS = 1, PTY_K_ROWS_INV = 2, PTY_K_PROBE = 3,
       PTY_K_REDUCE = 4, PTY_K_REFINE = 5, PTY_K_GRAD = 6, PTY_K_OTHER = 7,
       PTY_K_PATCH = 8, PTY_K_COUNT = 9 };
typedef struct {
  long long launches[PTY_K_COUNT];  /* kernel launches per kind */
  double ms[PTY_K_COUNT];           /* summed device time per kind (mode 1) */
  long long patches;                /* pattern updates processed */
} pty_stats;
int pty_profile(pty_handle* h, int mode);
int pty_get_stats(pty_handle* h, pty_stats* out, int reset);

/* Test hook for the error path of the staged passes.  With on = 1 the
 * mbarrier of every staged copy (the column pass's TMA loads, the inverse-row
 * pass's bulk copies) expects one more arrival than the copies make: each
 * copy still lands, but its bounded wait (0.2 s of the GPU's global timer)
 * runs out, the CTA records the time-out in the handle's status word, waits
 * (again bounded) for the copy it had in flight and leaves.  The next
 * synchronising call (pty_run_iterations with err_out, a copy-out to host
 * memory) returns PTY_ETIMEOUT and clears the word; the context stays usable,
 * but the object and probe of the interrupted iteration are undefined until
 * pty_set_data loads them again.  on = 0 restores normal operation.  Synchronises.  Nothing but tests should call this. */
int pty_debug_stall_copies(pty_handle* h, int on);

/* Differentiable forward model (bilinear crop at the exact float position,
 * Eqs. 1, 2, 4) with the amplitude loss
 *   L = sum_j sum_u (sqrt(sum_p |F(P_p o_j)|^2 + delta) - sqrt(I_j))^2
 * (delta >= 0 smooths the amplitude where the model is dark; 0 = plain).
 * O (Hy x Hx complex64), P (M x W x W complex64), pos (N x 2 float) and all
 * outputs are DEVICE pointers; the handle supplies the data I and scratch.
 * Every bilinear crop needs floor(pos) >= 0 and floor(pos) + W + 1 <= H
 * (else PTY_EDATA).  *loss is written on the device (one float).
 * pty_loss_grad also writes dL/dO (Hy x Hx), dL/dP (M x W x W) as
 * dL/dRe + i dL/dIm, and dL/dpos (N x 2); the far field is recomputed per
 * patch rather than stored.  dL/dO is accumulated group by group over
 * disjoint (W+1)-boxes, so results are bitwise repeatable. */
int pty_loss(pty_handle* h, const void* O, const void* P, const float* pos,
             float delta, float* loss);
int pty_loss_grad(pty_handle* h, const void* O, const void* P, const float* pos,
                  float delta, float* loss, void* gO, void* gP, float* gpos);

/* Model intensities sum_p |F{P_p o_j}|^2 (Eq. 4) for all j at the current
 * O, P and rounded positions: N*W*W float, detector-centred. */
int pty_model_intensities(pty_handle* h, float* dst, int mem_kind);

/* Model intensities, as pty_model_intensities, for callers that may not
 * allocate device memory at all (no counterpart in the paper: an interface
 * choice of this library).  Needs no handle: O (Hy x Hx), P (M x W x W,
 * complex64), pos (N x 2 float) and out (N x W x W float, detector-centred)
 * are caller-owned DEVICE pointers; work is queued on `stream`.  It calls no
 * allocator: its only intermediate lives in a fixed device array of
 * PTY_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * process exit.  One pattern needs M*W*W*8 bytes of it; larger requests fail
 * with PTY_EINVAL.  All calls share that array, so calls overlapping on the
 * GPU race; serialise them.  Every call resolves the array's device address
 * afresh (cudaGetSymbolAddress in the context current at the call; nothing
 * is cached, so a device reset or a caller's own driver context is safe).
 * The first call in a context may load the library's module and should come
 * before any stream capture.  A pattern whose crop box leaves the object is
 * written as NaN. */
#define PTY_NOALLOC_SCRATCH_BYTES ((size_t)6 << 20)
int pty_model_intensities_noalloc(const void* O, int Hy, int Hx, const void* P,
                                  int M, int W, const float* pos, int N,
                                  float* out, void* stream);

/* Batched form: many independent problems of uneven W, M and N run n_iter
 * M-rPIE iterations each inside ONE persistent, cooperative kernel launch
 * (captured in a CUDA graph).  A device task list interleaves the problems
 * pass by pass; each CTA takes the next task, waits (bounded by
 * timeout_ms on the GPU's global timer) until that problem has finished the
 * tasks its pass depends on, and runs it.  Results equal n_iter calls of
 * pty_run_iterations on each problem alone.  All problems use ds[0].stream.
 * pty_batch_problem lends the i-th problem's handle (set its data, read its
 * results; do not destroy it).  pty_batch_run returns PTY_ETIMEOUT if a wait
 * gave up (pty_batch_status then tells which problems are incomplete). */
typedef struct pty_batch pty_batch;
typedef struct {
  int split_rows;    /* tasks per row pass of a chunk (row blocks split)      */
  int split_cols;    /* tasks per patch of a column pass (column blocks split)*/
  int split_probe;   /* tasks per probe update                                */
  int timeout_ms;    /* bound on every device-side dependency wait            */
  int ctas;          /* cap on resident CTAs (0 = all that fit)               */
  int stall_problem; /* test hook: >= 0 gives that problem a dependency that
                        is never met, to exercise the bounded wait; -1 = off  */
} pty_batch_schedule;
int pty_batch_create(const pty_problem_desc* ds, int n, pty_batch** out);
int pty_batch_problem(pty_batch* b, int i, pty_handle** h);
int pty_batch_set_schedule(pty_batch* b, const pty_batch_schedule* s);
int pty_batch_run(pty_batch* b, int n_iter, const pty_rpie_params* p);
int pty_batch_status(pty_batch* b, int* per_problem);
int pty_batch_destroy(pty_batch* b);

/* Orthogonalise the probe modes in place (between iterations; the paper's
 * mixed state, Eq. 4, after the multimode ePIE of Thibault & Menzel 2013):
 * with the Gram matrix G_kl = sum_r conj(P_k(r)) P_l(r) = V diag(w) V^H
 * (w decreasing), P'_m = sum_k V_km P_k.  The new modes are mutually
 * orthogonal, sum_r |P'_m|^2 = w_m, and the density matrix
 * sum_k P_k(r) conj(P_k(r')) is unchanged.  Each eigenvector's phase is fixed
 * by making its largest-magnitude entry (the first on ties) real and
 * positive.  G is reduced on the GPU in double precision, the M x M
 * eigenproblem solved on the host (double, cyclic Jacobi), V applied on the
 * GPU.  power_out (host, M doubles, may be NULL) receives w.  Synchronises. */
int pty_orthogonalize_probe(pty_handle* h, double* power_out);

/* Host-only Hermitian eigensolver used by pty_orthogonalize_probe (no GPU
 * needed): A is M x M (M <= 16) complex, row-major, interleaved (re, im)
 * doubles; w receives the eigenvalues in decreasing order, V (M x M, same
 * layout) the eigenvectors as columns, phases fixed as above. */
int pty_hermitian_eig(int M, const double* A, double* w, double* V);

/* Host-only greedy grouping (no GPU needed): positions pos (N*2, host),
 * boxes of side W, optional order (NULL = index order), max_group (0 =
 * unlimited).  Writes group_ptr (capacity N+1), group_pos (N), *n_groups.
 * Each position goes to the first group with no overlapping box. */
int pty_group_positions(const float* pos, int N, int W, int max_group,
                        const int32_t* order, int32_t* group_ptr,
                        int32_t* group_pos, int* n_groups);

/* Unnormalised 2-D DFT of `batch` W x W complex64 arrays, in place, device
 * memory, through the same line FFTs the reconstruction uses (a check of
 * the FFT alone).  inverse = 0: exp(-2 pi i ...), 1: exp(+2 pi i ...). */
int pty_fft2(void* data, int W, int batch, int inverse, void* stream);

/* Measured FP32 FMA throughput of the current device in TFLOP/s (eight
 * independent FMA chains per thread, 8 CTAs of 256 threads per SM, best of
 * three timed launches): the measured counterpart of the nominal FP32 peak
 * the passes' roofline uses.  Allocates and frees about 1 MB; synchronises. */
int pty_measure_fp32_peak(double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* PTY_H_ */
