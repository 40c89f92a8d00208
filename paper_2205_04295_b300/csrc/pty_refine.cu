// XCORR_A / XCORR_B registration and the Adam position step (Adam-based
// position refinement section of Guzzi et al., arXiv 2205.04295; Eqs. 8-9,
// Algorithm 1, the two switch positions of Fig. 2; registration after
// Guizar-Sicairos, Thurman & Fienup, Opt. Lett. 33, 156, 2008).
//
// For each patch of a group, after pass C, the scratch holds
//   XCORR_A: plane M     : row DFTs of o_j   (crop before the update; pass A)
//            plane M + 1 : row DFTs of o'_j  (refined crop; pass C)
//   XCORR_B: planes M, M + 1: the model intensity sum_p |Psi_p|^2 and the
//            counts I_j (real images, unshifted; pass B), turned into row
//            DFTs by xcorrb_rows
// and the same correlation passes follow:
// xcorr_cols : column DFTs of both planes -> A = F(o_j), B = F(o'_j);
//              X = B conj(A) is stored in plane M; inverse column DFTs of X
//              into plane M+1.
// xcorr_rows : inverse row DFTs of plane M+1 -> c = F^-1 X (unnormalised);
//              per row block the largest |c|^2 and its first row-major index.
// updft      : coarse peak (s_y, s_x) wrapped to [-W/2, W/2); the
//              cross-correlation re-evaluated on the K x K grid
//              s + (k - K/2)/U as E_r X E_c; its first maximum gives the
//              shift s_j; the stored measurement is g_j = -s_j.
// adam       : one Adam step per position with g_j as the gradient, then the
//              position is clamped so that its crop stays inside the object.
//
// The phase of every matrix-DFT entry is an exact integer multiple of
// 2 pi / (U W): entry (v, k) of E_c is root[(v_s (U s_x + k - K/2)) mod (U W)]
// with v_s the signed frequency; the roots come from a host table.
#include "pty_copy.cuh"
#include "pty_fft.cuh"
#include "pty_internal.h"
#include "pty_pdl.cuh"
#include "pty_tc.cuh"

#include <algorithm>
#include <cmath>

namespace pty {

namespace {

// larger value wins; equal values: smaller index wins (first in row-major order)
PTY_D void best_merge(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

PTY_D void warp_best(float& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    best_merge(v, i, v2, i2);
  }
}

// Block-wide best (value, index); every thread gets it.  Contains barriers.
PTY_D void block_best(float& v, int& i, float* rv, int* ri) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  warp_best(v, i);
  __syncthreads();
  if (l == 0) {
    rv[w] = v;
    ri[w] = i;
  }
  __syncthreads();
  v = rv[0];
  i = ri[0];
  for (int k = 1; k < nw; ++k) best_merge(v, i, rv[k], ri[k]);
}

PTY_D int wrap_shift(int i, int W) { return i >= W / 2 ? i - W : i; }
PTY_D int modp(long long a, int m) {
  long long r = a % m;
  return (int)(r < 0 ? r + m : r);
}

// ------------------------------------------------------------ xcorr_cols
template <int W>
__global__ void __launch_bounds__(256)
k_xcorr_cols(float2* __restrict__ scratch, int npl, int M, int CB,
             const float2* __restrict__ tw_g) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  pdl_trigger();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  pdl_wait();  // both crops' row DFTs come from the passes
  const int lp = blockIdx.y, c0 = blockIdx.x * CB;
  const int c = threadIdx.x % CB, lane = threadIdx.x / CB;
  const bool act = lane < G::L;
  float2* colA = scratch + ((size_t)lp * npl + M) * W * W + c0 + c;
  float2* colB = colA + (size_t)W * W;
  float2* lbuf = tbuf + c * G::LP;
  // the first crop's column; the second one is loaded once the first is
  // transformed, so that only one column is held in registers at a time
  float2 v[G::N1];
  if (act && lane < G::N2) {
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = colA[(size_t)(G::N2 * n1 + lane) * W];
  }
  __syncthreads();
  // A = F(o_j): the column DFTs of plane M (its row DFTs come from pass A)
  if (act && lane < G::N2) fwd_step1<W>(v, lane, tw, lbuf);
  if (act && lane < G::N2) {
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = colB[(size_t)(G::N2 * n1 + lane) * W];
  }
  __syncthreads();
  float2 za[G::N2];
  if (act && lane < G::N1) fwd_step3<W>(za, lane, lbuf);
  __syncthreads();
  // B = F(o'_j)
  if (act && lane < G::N2) fwd_step1<W>(v, lane, tw, lbuf);
  __syncthreads();
  float2 z[G::N2];
  if (act && lane < G::N1) {
    fwd_step3<W>(z, lane, lbuf);
#pragma unroll
    for (int k2 = 0; k2 < G::N2; ++k2) {
      const size_t u = lane + G::N1 * k2;
      const float2 X = cmulc(z[k2], za[k2]);  // B conj(A)
      colA[u * W] = X;
      z[k2] = X;
    }
  }
  __syncthreads();  // all transposes read before they are overwritten
  if (act && lane < G::N1) inv_stepA<W>(z, lane, tw, lbuf);
  __syncthreads();
  if (act && lane < G::N2) {
    inv_stepB<W>(v, lane, lbuf);
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) colB[(size_t)(G::N2 * n1 + lane) * W] = v[n1];
  }
}

// ------------------------------------------------------------ xcorrb_rows
// Forward row DFTs, in place, of consecutive planes starting at plane M (the
// kernel's M): XCORR_B's two real images pass B left in planes M (model
// intensity) and M + 1 (counts), or XCORR_A's refined crop, which pass C
// leaves untransformed in plane M + 1.  The correlation passes then take them
// as they take the crops' row DFTs.  A CTA's RX lines are rows of the block
// of consecutive planes.
template <int W>
__global__ void __launch_bounds__(256)
k_xcorrb_rows(float2* __restrict__ scratch, int npl, int M, int RX,
              const float2* __restrict__ tw_g) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  pdl_trigger();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  pdl_wait();  // the images come from the column pass (XCORR_B) or pass C (XCORR_A)
  __syncthreads();
  const int lp = blockIdx.y, r0 = blockIdx.x * RX;
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < RX;
  float2* lbuf = tbuf + line * G::LP;
  float2* row = scratch + (((size_t)lp * npl + M) * W + r0 + (act ? line : 0)) * W;
  if (act && lane < G::N2) {
    float2 v[G::N1];
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = row[G::N2 * n1 + lane];
    fwd_step1<W>(v, lane, tw, lbuf);
  }
  __syncthreads();
  if (act && lane < G::N1) {
    float2 z[G::N2];
    fwd_step3<W>(z, lane, lbuf);
#pragma unroll
    for (int k2 = 0; k2 < G::N2; ++k2) row[lane + G::N1 * k2] = z[k2];
  }
}

// ------------------------------------------------------------ xcorr_rows
template <int W>
__global__ void __launch_bounds__(256)
k_xcorr_rows(const float2* __restrict__ scratch, int npl, int M, int RX,
             const float2* __restrict__ tw_g, float* __restrict__ cval,
             int* __restrict__ cidx) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  __shared__ float rv[32];
  __shared__ int ri[32];
  pdl_trigger();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  pdl_wait();  // X comes from the correlation column pass
  __syncthreads();
  const int lp = blockIdx.y, r0 = blockIdx.x * RX;
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < RX;
  float2* lbuf = tbuf + line * G::LP;
  const float2* row = scratch + (((size_t)lp * npl + M + 1) * W + r0 + (act ? line : 0)) * W;
  if (act && lane < G::N1) {
    float2 z[G::N2];
#pragma unroll
    for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = row[lane + G::N1 * k2];
    inv_stepA<W>(z, lane, tw, lbuf);
  }
  __syncthreads();
  float best = -1.f;
  int bi = 0x7fffffff;
  if (act && lane < G::N2) {
    float2 v[G::N1];
    inv_stepB<W>(v, lane, lbuf);
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1)
      best_merge(best, bi, cabs2(v[n1]), (r0 + line) * W + G::N2 * n1 + lane);
  }
  block_best(best, bi, rv, ri);
  if (threadIdx.x == 0) {
    cval[(size_t)lp * gridDim.x + blockIdx.x] = best;
    cidx[(size_t)lp * gridDim.x + blockIdx.x] = bi;
  }
}

// ------------------------------------------------------------ updft
// The fine grid is evaluated as c_up = E_r X E_c in two kernels:
//   updft_part : CTA (row block of RB rows of X, patch): T = X_rows E_c
//                (RB x K) and the block's share E_r[:, rows] T (K x K),
//                written as a partial sum;
//   updft_final: per patch, the partial sums added in block order, |c_up|^2,
//                first maximum in row-major order -> shift.
// The phase of every entry is an exact multiple of 2 pi / (U W), read from
// the root table staged in shared memory.  T is register-tiled: a thread
// accumulates 2 rows x 4 fine-grid columns, and the 32 threads of a warp
// share the columns, so each root lookup is a broadcast.

PTY_D void coarse_peak(const float* cval, const int* cidx, int lp, int nparts, int W,
                       int& sy, int& sx, float* rv, int* ri) {
  float b = -1.f;
  int bi = 0x7fffffff;
  for (int e = threadIdx.x; e < nparts; e += blockDim.x)
    best_merge(b, bi, cval[(size_t)lp * nparts + e], cidx[(size_t)lp * nparts + e]);
  block_best(b, bi, rv, ri);
  sy = wrap_shift(bi / W, W);
  sx = wrap_shift(bi % W, W);
}

// acc += a b, complex, as four fused multiply-adds
PTY_D void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

template <int W>
__global__ void __launch_bounds__(512)
k_updft_part(const float2* __restrict__ scratch, int npl, int M, int nparts,
             const float* __restrict__ cval, const int* __restrict__ cidx,
             const float2* __restrict__ roots_g, int U, int K, int RB,
             float2* __restrict__ part) {
  extern __shared__ float4 smem4[];
  const int UW = U * W;
  constexpr int XP = W + 1;                  // padded row pitch of the X block
  const int KP = (K + 3) / 4 * 4;            // columns padded to whole tiles
  float2* E = reinterpret_cast<float2*>(smem4);  // [W][KP]: this patch's E_c
  float2* Xs = E + W * KP;                   // [RB][W + 1]
  float2* T = Xs + RB * XP;                  // [RB][KP]
  float2* Er = T + RB * KP;                  // [K][RB]: this block's E_r columns
  __shared__ float rv[32];
  __shared__ int ri[32];
  const int lp = blockIdx.y, u0 = blockIdx.x * RB;
  const float2* X = scratch + ((size_t)lp * npl + M) * W * W + (size_t)u0 * W;
  pdl_trigger();
  pdl_wait();  // X and the coarse peaks come from the correlation passes
  // all staging is asynchronous (cp.async): no thread waits on a load
  // before issuing the next one
  for (int e = threadIdx.x; e < RB * W; e += blockDim.x) {
    const int r = e / W, v = e - r * W;
    cp_async<8>(Xs + r * XP + v, X + (size_t)r * W + v);
  }
  int sy, sx;
  coarse_peak(cval, cidx, lp, nparts, W, sy, sx, rv, ri);  // contains barriers
  const int half = K / 2;
  // E[v][k] = root[(v_s (U sx + k - half)) mod UW]: a thread fills one column
  // over a run of 32 frequencies (runs never straddle v = W/2), stepping the
  // index instead of reducing a product per entry
  for (int t = threadIdx.x; t < KP * (W / 32 + (W % 32 != 0)); t += blockDim.x) {
    const int k = t % KP, v0 = (t / KP) * 32, v1 = min(W, v0 + 32);
    const int a = modp((long long)U * sx + min(k, K - 1) - half, UW);
    int n = -1;
    for (int v = v0; v < v1; ++v) {
      if (n < 0 || v == W / 2) {
        n = modp((long long)(v < W / 2 ? v : v - W) * a, UW);
      } else {
        n += a;
        if (n >= UW) n -= UW;
      }
      cp_async<8>(E + v * KP + k, roots_g + n);
    }
  }
  for (int t = threadIdx.x; t < K * RB; t += blockDim.x) {
    const int k1 = t / RB, r = t - k1 * RB, u = u0 + r;
    const int b = modp((long long)U * sy + k1 - half, UW);
    cp_async<8>(Er + t, roots_g + modp((long long)(u < W / 2 ? u : u - W) * b, UW));
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  // T[r][k] = sum_v X[u0 + r][v] E[v][k]; a thread holds 1 row x 4 columns,
  // a warp 32 rows of the same columns (E reads are broadcasts)
  const int nkt = KP / 4;
  for (int tile = threadIdx.x; tile < RB * nkt; tile += blockDim.x) {
    const int r0 = tile % RB, k0 = 4 * (tile / RB);
    float2 c0[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c0[q] = make_float2(0.f, 0.f);
    const float2* x0 = Xs + r0 * XP;
    const float4* ev = reinterpret_cast<const float4*>(E + k0);
#pragma unroll 4
    for (int v = 0; v < W; ++v) {
      const float2 p0 = x0[v];
      const float4 ea = ev[(v * KP) / 2], eb = ev[(v * KP) / 2 + 1];
      cfma(c0[0], p0, make_float2(ea.x, ea.y));
      cfma(c0[1], p0, make_float2(ea.z, ea.w));
      cfma(c0[2], p0, make_float2(eb.x, eb.y));
      cfma(c0[3], p0, make_float2(eb.z, eb.w));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) T[r0 * KP + k0 + q] = c0[q];
  }
  __syncthreads();
  // share of this row block: sum_{r} E_r[k1][u0 + r] T[r][k2]
  float2* dst = part + ((size_t)lp * gridDim.x + blockIdx.x) * K * K;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int k1 = e / K, k2 = e - k1 * K;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < RB; ++r) cfma(acc, Er[k1 * RB + r], T[r * KP + k2]);
    dst[e] = acc;
  }
}

// Sum of a patch's fine-grid shares in block order, |c_up|^2, its first
// maximum in row-major order and the gap to the second best; writes the
// measurement g_j = -shift of pattern j.  Contains barriers.
PTY_D void updft_finish(int lp, int j, int sy, int sx, int nblocks, int U, int K,
                        const float2* part, float* shift, float* gap, float* rv, int* ri) {
  const int half = K / 2;
  float best = -1.f, second = -1.f;
  int bi = 0x7fffffff;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < nblocks; ++b)  // fixed order
      acc = cadd(acc, __ldcg(part + ((size_t)lp * nblocks + b) * K * K + e));
    const float m = cabs2(acc);
    if (m > best) {
      second = fmaxf(second, best);
      best = m;
      bi = e;
    } else {
      second = fmaxf(second, m);
    }
  }
  float gb = best;
  int gbi = bi;
  block_best(gb, gbi, rv, ri);
  float s2 = (bi == gbi) ? second : best;  // best of this thread that is not the winner
  __syncthreads();
  {
    int dummy = 0;
    block_best(s2, dummy, rv, ri);
  }
  if (threadIdx.x == 0) {
    const int k1 = gbi / K, k2 = gbi % K;
    const float y = (float)sy + (float)(k1 - half) / (float)U;
    const float x = (float)sx + (float)(k2 - half) / (float)U;
    shift[2 * j] = -y;
    shift[2 * j + 1] = -x;
    gap[j] = gb > 0.f ? (gb - fmaxf(s2, 0.f)) / gb : 0.f;
  }
}

// ------------------------------------------------------------ updft_tc
// Tensor-core form of updft_part (tcgen05, kind::tf32, 3xTF32 split): CTA
// (tile of 128 rows of X, patch).  T = X_rows E_c is taken on the
// 5th-generation tensor cores as one real GEMM pair,
//   [Re T | Im T] = Xr [Ecr | Eci] + Xi [-Eci | Ecr]   (M 128, N 64, K = W).
// Every operand is split x = hi + lo into TF32 parts and each product is
// hi hi + hi lo + lo hi, which keeps about 21 bits of each operand
// (FP32-level results).  The hi and lo parts of an E_c operand are stacked
// along N (rows 0-63 hi, 64-127 lo), so per K step one N = 128 MMA takes
// X_hi [B_hi | B_lo] and one N = 64 MMA adds X_lo B_hi into the first half:
// the 128 x 128 FP32 accumulator in TMEM holds [hi-hi + lo-hi | hi-lo]
// products, added at read-out.
//
// Pipeline over chunks of 16 columns of X: each thread loads its 8 values of
// the next chunk into registers while the current one is split; a chunk is
// split into four K-major planes (Xr hi, Xr lo, Xi hi, Xi lo) and the
// matching chunk of the two stacked E_c operands into two more, in one of
// two plane buffers (96 KB: two CTAs per SM, whose phases interleave); one thread issues the chunk's 8
// MMAs and commits them to that buffer's mbarrier, and the CTA goes on to
// split the next chunk into the other buffer while they run (a buffer is
// refilled once its mbarrier says the MMAs that read it are done; every
// wait is bounded).  The phases exp(2 pi i n / (U W)) come from the root
// table through L1; their indices are stepped in 32-bit integers.  The block's share E_r[:, rows] T (K x K)
// is then taken on the FP32 cores (2 x 2 outputs per thread) from T copied
// to shared memory, and updft_final adds the shares.  Rows past W (W < 128,
// or the second tile at W = 192) are zero.
constexpr int kTcRows = 128;                  // M of the MMA: rows of X per CTA
constexpr int kTcKc = 16;                     // columns of X (index v) per chunk
constexpr int kTcN = 32;                      // fine-grid points held (K <= 32)
constexpr int kTcTPitch = kTcN + 1;           // complex per row of T in shared memory
constexpr int kTcAPlane = kTcRows * kTcKc * 4;    // bytes of one A plane (128 x 16)
constexpr int kTcBPlane = 4 * kTcN * kTcKc * 4;   // bytes of one stacked B plane (128 x 16)
constexpr int kTcBuf = 4 * kTcAPlane + 2 * kTcBPlane;  // one set of operand planes
constexpr int kTcSBO = (kTcKc / 4) * 128;         // bytes between 8-row groups
constexpr int kTcFixed = 2 * kTcBuf + 128;  // two plane buffers: two CTAs per SM
static_assert(kTcRows * kTcTPitch * 8 <= kTcBuf, "T reuses the second plane buffer");
static_assert(kTcN * kTcRows * 8 <= kTcBuf, "E_r reuses the first plane buffer");

// Byte offset of element (row, k) in a K-major, no-swizzle plane of kTcKc
// columns: core matrices (8 rows x 4 values, 128 bytes) with the K-adjacent
// ones contiguous (LBO = 128) and the row-adjacent ones kTcKc / 4 apart
// (SBO = kTcSBO).
__device__ __forceinline__ int tc_off(int row, int k) {
  return ((row >> 3) * (kTcKc / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ int modp32(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}
__device__ __forceinline__ void split4(const float* x, float4& hi, float4& lo) {
  tf32_split(x[0], hi.x, lo.x);
  tf32_split(x[1], hi.y, lo.y);
  tf32_split(x[2], hi.z, lo.z);
  tf32_split(x[3], hi.w, lo.w);
}

template <int W>
__global__ void __launch_bounds__(256, 2)
k_updft_tc(const float2* __restrict__ scratch, int npl, int M, int nparts,
           const float* __restrict__ cval, const int* __restrict__ cidx,
           const float2* __restrict__ roots_g, int U, int K, float2* __restrict__ part,
           const int* __restrict__ ids, int* __restrict__ done, float* __restrict__ shift,
           float* __restrict__ gap, int* __restrict__ err) {
  extern __shared__ float4 smem4[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tslot;
  __shared__ float rv[32];
  __shared__ int ri[32];
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem4) + 127) &
                                       ~static_cast<uintptr_t>(127));
  char* pl = base;                                  // 2 x (Xr hi, Xr lo, Xi hi, Xi lo, B1, B2)
  const float2* roots = roots_g;                    // U W roots, read through L1
  float2* T = reinterpret_cast<float2*>(pl + kTcBuf);  // [128][kTcTPitch] after the MMAs
  float2* Er = reinterpret_cast<float2*>(pl);       // [K][128] after the MMAs

  const int lp = blockIdx.y, u0 = blockIdx.x * kTcRows;
  const int nrows = min(kTcRows, W - u0);
  const int UW = U * W, half = K / 2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const float2* X = scratch + ((size_t)lp * npl + M) * W * W + (size_t)u0 * W;
  constexpr int nch = W / kTcKc;
  constexpr unsigned long long kLimit = 200000000ull;  // 0.2 s of the global timer
  pdl_trigger();
  if (warp == 0) tmem_alloc(&tslot, 128);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  pdl_wait();  // X and the coarse peaks come from the correlation passes
  // A thread's X values of a chunk: row m = tid mod 128, the chunk's columns
  // 4q .. 4q + 3 for q = 2 (tid / 128) + 0, 1 (8 complex, contiguous; zero past
  // the last row), loaded into registers one chunk ahead.
  const int xm = tid & (kTcRows - 1);
  const bool xrow = xm < nrows;
  const float4* xsrc = reinterpret_cast<const float4*>(X + (size_t)(xrow ? xm : 0) * W +
                                                       8 * (tid >> 7));
  // two chunks ahead: X comes from HBM (a batch's planes exceed L2)
  float4 xn[4], xn2[4];
  auto fetch = [&](float4* dst, int c) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      dst[i] = (c < nch && xrow) ? __ldcs(xsrc + c * (kTcKc / 2) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  fetch(xn, 0);
  fetch(xn2, 1);
  int sy, sx;
  coarse_peak(cval, cidx, lp, nparts, W, sy, sx, rv, ri);  // contains barriers
  tc_fence_after_sync();
  const uint32_t tm = tslot;
  // E_c entry (v, k) = root[(v_s a_k) mod UW], a_k = U s_x + k - K/2; threads
  // 0-127 write the operand rows of fine-grid point kq, columns vq .. vq + 3
  // (a warp covers 8 consecutive kq and the 4 column groups: conflict-free)
  const int kq = 8 * (warp & 3) + (tid & 7), vq = 4 * ((tid & 31) >> 3);
  const int a_k = modp32(U * sx + kq - half, UW);
  // this thread's four E_c roots of a chunk, loaded one chunk ahead (the
  // table is read through L1, which two CTAs' shared memory leaves small)
  auto roots_of = [&](int c, float2* w) {
    if (tid < 4 * kTcN && kq < K && c < nch) {
      const int v0 = c * kTcKc + vq;  // 4 | W / 2: the four columns share a sign
      int n = modp32((v0 < W / 2 ? v0 : v0 - W) * a_k, UW);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        w[e] = __ldg(roots + n);
        n += a_k;
        if (n >= UW) n -= UW;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) w[e] = make_float2(0.f, 0.f);
    }
  };
  float2 wn[4];
  roots_of(0, wn);
  const uint32_t id128 = tc_idesc_tf32(kTcRows, 4 * kTcN, false);
  const uint32_t id64 = tc_idesc_tf32(kTcRows, 2 * kTcN, false);
  // descriptors of buffer 0; the other planes differ only in the start field
  // (address / 16, well inside its 14 bits)
  const uint64_t d0 = tc_smem_desc(pl, 128, kTcSBO);
  unsigned ph = 0u;  // bit b: parity of the next completion of mbar[b]
  auto fail = [&](bool mine, int b) {
    if (tid == 0) atomicExch(err, 1);
    if (mine) mbar_wait_bounded(&mbar[b], ((ph >> b) & 1u) ^ 1u, kLimit);  // the MMAs in flight
    cp_async_wait<0>();
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, 128);
  };
  for (int c = 0; c < nch; ++c) {
    const int b = c & 1;
    float4 xc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xc[i] = xn[i];
      xn[i] = xn2[i];
    }
    fetch(xn2, c + 2);  // in flight while this chunk and the next are split
    bool ok = true;
    if (c >= 2) {  // the MMAs of chunk c - 2 still read plane buffer b
      ok = mbar_wait_bounded(&mbar[b], (ph >> b) & 1u, kLimit);
      ph ^= 1u << b;
    }
    if (__syncthreads_or(!ok)) {
      fail(!ok, b);
      return;
    }
    char* Ap = pl + b * kTcBuf;
    char* Bp = Ap + 4 * kTcAPlane;
    {  // X split: thread -> row m, core-matrix columns q = 2 (tid / 128) + 0..1
      const int m = xm;
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * (tid >> 7) + qq;
        const float4 x0 = xc[2 * qq];
        const float4 x1 = xc[2 * qq + 1];
        const float re[4] = {x0.x, x0.z, x1.x, x1.z}, im[4] = {x0.y, x0.w, x1.y, x1.w};
        float4 rh, rl, ih, il;
        split4(re, rh, rl);
        split4(im, ih, il);
        const int off = tc_off(m, 4 * q);
        *reinterpret_cast<float4*>(Ap + off) = rh;
        *reinterpret_cast<float4*>(Ap + kTcAPlane + off) = rl;
        *reinterpret_cast<float4*>(Ap + 2 * kTcAPlane + off) = ih;
        *reinterpret_cast<float4*>(Ap + 3 * kTcAPlane + off) = il;
      }
    }
    if (tid < 4 * kTcN) {  // E_c split: B1 = [Ecr | Eci], B2 = [-Eci | Ecr], lo parts 64 rows down
      float cr[4], ci[4], nci[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        cr[e] = wn[e].x;  // zero past K
        ci[e] = wn[e].y;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) nci[e] = -ci[e];
      float4 rh, rl, ih, il, nh, nl;
      split4(cr, rh, rl);
      split4(ci, ih, il);
      split4(nci, nh, nl);
      const int o1 = tc_off(kq, vq), o2 = tc_off(kTcN + kq, vq);
      const int l1 = tc_off(2 * kTcN + kq, vq), l2 = tc_off(3 * kTcN + kq, vq);
      char* B1 = Bp;
      char* B2 = Bp + kTcBPlane;
      *reinterpret_cast<float4*>(B1 + o1) = rh;
      *reinterpret_cast<float4*>(B1 + o2) = ih;
      *reinterpret_cast<float4*>(B1 + l1) = rl;
      *reinterpret_cast<float4*>(B1 + l2) = il;
      *reinterpret_cast<float4*>(B2 + o1) = nh;
      *reinterpret_cast<float4*>(B2 + o2) = rh;
      *reinterpret_cast<float4*>(B2 + l1) = nl;
      *reinterpret_cast<float4*>(B2 + l2) = rl;
    }
    roots_of(c + 1, wn);  // in flight while this chunk's MMAs are issued and run
    fence_proxy_async();  // the planes, written through the generic proxy, go to the MMA
    __syncthreads();
    if (tid == 0) {
      tc_fence_after_sync();
      const uint64_t db = d0 + (uint64_t)((b * kTcBuf) >> 4);
#pragma unroll
      for (int s = 0; s < kTcKc / 8; ++s) {
        const uint64_t ds = db + (uint64_t)((s * 256) >> 4);
        const uint64_t xrh = ds, xrl = ds + (kTcAPlane >> 4);
        const uint64_t xih = ds + ((2 * kTcAPlane) >> 4), xil = ds + ((3 * kTcAPlane) >> 4);
        const uint64_t b1 = ds + ((4 * kTcAPlane) >> 4);
        const uint64_t b2 = ds + ((4 * kTcAPlane + kTcBPlane) >> 4);
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        tc_mma_tf32(tm, xrh, b1, id128, acc);  // Xr hi [B1 hi | B1 lo]
        tc_mma_tf32(tm, xrl, b1, id64, 1u);    // Xr lo B1 hi
        tc_mma_tf32(tm, xih, b2, id128, 1u);   // Xi hi [B2 hi | B2 lo]
        tc_mma_tf32(tm, xil, b2, id64, 1u);    // Xi lo B2 hi
      }
      tc_commit(&mbar[b]);
    }
  }
  {  // the last chunk's commit covers every MMA issued before it
    const int b = (nch - 1) & 1;
    const bool ok = mbar_wait_bounded(&mbar[b], (ph >> b) & 1u, kLimit);
    ph ^= 1u << b;
    if (__syncthreads_or(!ok)) {
      fail(!ok, b);
      return;
    }
  }
  cp_async_wait<0>();
  tc_fence_after_sync();
  {  // T -> shared memory: warps 0-3 Re T, 4-7 Im T of row 32 (warp % 4) + lane,
     // each the sum of the hi-hi + lo-hi and the hi-lo accumulator halves
    float v[kTcN], w[kTcN];
    const uint32_t ta = tm + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * kTcN);
    tmem_ld32(ta, v);
    tmem_ld32(ta + 2 * kTcN, w);
    const int m = 32 * (warp & 3) + (tid & 31);
    float* Tf = reinterpret_cast<float*>(T) + 2 * m * kTcTPitch + (warp >> 2);
#pragma unroll
    for (int k = 0; k < kTcN; ++k) Tf[2 * k] = v[k] + w[k];
  }
  // this block's E_r columns: Er[k1][r] = root[(u_s (U s_y + k1 - K/2)) mod UW]
  for (int t = tid; t < K * kTcRows; t += blockDim.x) {
    const int k1 = t / kTcRows, r = t - k1 * kTcRows, u = u0 + r;
    const int bk = modp32(U * sy + k1 - half, UW);
    Er[t] = r < nrows ? roots[modp32((u < W / 2 ? u : u - W) * bk, UW)] : make_float2(0.f, 0.f);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc(tm, 128);
  }
  // share of this row block: sum_r E_r[k1][u0 + r] T[r][k2], 2 x 2 outputs per thread
  float2* dst = part + ((size_t)lp * gridDim.x + blockIdx.x) * K * K;
  const int nb = (K + 1) / 2;
  if (tid < nb * nb) {
    const int k1 = 2 * (tid / nb), k2 = 2 * (tid % nb);
    const bool y1 = k1 + 1 < K, x1 = k2 + 1 < K;
    const float2* e0 = Er + k1 * kTcRows;
    const float2* e1 = Er + (y1 ? k1 + 1 : k1) * kTcRows;
    float2 c00 = make_float2(0.f, 0.f), c01 = c00, c10 = c00, c11 = c00;
#pragma unroll 4
    for (int r = 0; r < nrows; ++r) {
      const float2 a0 = e0[r], a1 = e1[r];
      const float2 t0 = T[r * kTcTPitch + k2], t1 = T[r * kTcTPitch + k2 + 1];
      cfma(c00, a0, t0);
      cfma(c01, a0, t1);
      cfma(c10, a1, t0);
      cfma(c11, a1, t1);
    }
    dst[k1 * K + k2] = c00;
    if (x1) dst[k1 * K + k2 + 1] = c01;
    if (y1) dst[(k1 + 1) * K + k2] = c10;
    if (y1 && x1) dst[(k1 + 1) * K + k2 + 1] = c11;
  }
  // the last of the patch's CTAs to finish adds the shares (block order) and
  // takes the argmax; done[lp] counts the finished CTAs and is left at zero
  __shared__ int s_last;
  __threadfence();  // this CTA's share is visible before it is counted
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&done[lp], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (tid == 0) done[lp] = 0;
    updft_finish(lp, ids[lp], sy, sx, gridDim.x, U, K, part, shift, gap, rv, ri);
  }
}

__global__ void __launch_bounds__(256)
k_updft_final(const int* __restrict__ ids, int W, int nblocks, int nparts,
              const float* __restrict__ cval, const int* __restrict__ cidx, int U, int K,
              const float2* __restrict__ part, float* __restrict__ shift,
              float* __restrict__ gap) {
  __shared__ float rv[32];
  __shared__ int ri[32];
  pdl_trigger();
  pdl_wait();  // the partial sums come from updft_part
  const int lp = blockIdx.x;
  int sy, sx;
  coarse_peak(cval, cidx, lp, nparts, W, sy, sx, rv, ri);
  updft_finish(lp, ids[lp], sy, sx, nblocks, U, K, part, shift, gap, rv, ri);
}

// U <= 1: the coarse peak alone.
__global__ void k_coarse_only(const int* __restrict__ ids, int nparts, int W,
                              const float* __restrict__ cval, const int* __restrict__ cidx,
                              float* __restrict__ shift, float* __restrict__ gap) {
  __shared__ float rv[32];
  __shared__ int ri[32];
  const int lp = blockIdx.x, j = ids[lp];
  float b = -1.f;
  int bi = 0x7fffffff;
  for (int e = threadIdx.x; e < nparts; e += blockDim.x)
    best_merge(b, bi, cval[(size_t)lp * nparts + e], cidx[(size_t)lp * nparts + e]);
  block_best(b, bi, rv, ri);
  if (threadIdx.x == 0) {
    shift[2 * j] = -(float)wrap_shift(bi / W, W);
    shift[2 * j + 1] = -(float)wrap_shift(bi % W, W);
    gap[j] = 1.f;
  }
}

// ------------------------------------------------------------ adam
__global__ void k_adam(float* __restrict__ pos, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int N, float lr, float b1, float b2,
                       float eps, float bc1, float bc2, float max_step, float ymax,
                       float xmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * N) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  float step = lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  if (max_step > 0.f) step = fminf(fmaxf(step, -max_step), max_step);
  const float hi = (i & 1) ? xmax : ymax;
  pos[i] = fminf(fmaxf(pos[i] + step, 0.f), hi);
}

int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

}  // namespace

#define PTY_DISPATCH_W(W, ...)                                 \
  switch (W) {                                                 \
    case 32: { constexpr int WW = 32; __VA_ARGS__; } break;     \
    case 64: { constexpr int WW = 64; __VA_ARGS__; } break;     \
    case 96: { constexpr int WW = 96; __VA_ARGS__; } break;     \
    case 128: { constexpr int WW = 128; __VA_ARGS__; } break;   \
    case 192: { constexpr int WW = 192; __VA_ARGS__; } break;   \
    case 256: { constexpr int WW = 256; __VA_ARGS__; } break;   \
    default: return cudaErrorInvalidValue;                     \
  }

template <int W> static void refgeo_fill(RefGeo& g) {
  using G = Line<W>;
  g.CBX = std::min(16, pow2_floor(256 / G::L));
  while ((W / 2) % g.CBX) g.CBX /= 2;
  g.RX = std::min(W, pow2_floor(256 / G::L));
  while (W % g.RX) g.RX /= 2;
  g.smX = (size_t)(W + g.CBX * G::LP) * sizeof(float2);
  g.smR = (size_t)(W + g.RX * G::LP) * sizeof(float2);
}

RefGeo make_refgeo(int W, int U, bool tc) {
  RefGeo g{};
  g.W = W;
  g.U = std::max(1, U);
  g.K = (int)std::ceil(1.5 * g.U);
  g.tc = tc && g.U > 1 && g.K <= kTcN && (size_t)kTcFixed <= (size_t)smem_optin() - 1024;
  switch (W) {
    case 32: refgeo_fill<32>(g); break;
    case 64: refgeo_fill<64>(g); break;
    case 96: refgeo_fill<96>(g); break;
    case 128: refgeo_fill<128>(g); break;
    case 192: refgeo_fill<192>(g); break;
    default: refgeo_fill<256>(g); break;
  }
  // the most X rows per CTA (64, 32 or 16, at most W/2) whose tables fit
  const int KP = (g.K + 3) / 4 * 4;
  for (g.RB = std::min(64, std::max(16, W / 2)); ; g.RB /= 2) {
    g.smU = (size_t)(W * KP + g.RB * (W + 1) + g.RB * KP + g.K * g.RB) * sizeof(float2);
    if (g.smU <= (size_t)smem_optin() - 1024 || g.RB <= 16) break;
  }
  return g;
}

cudaError_t set_refine_smem(const RefGeo& g) {
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(g.W, {
    e = allow_max_smem((const void*)k_xcorr_cols<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_xcorr_rows<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_xcorrb_rows<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_updft_part<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_updft_tc<WW>);
  });
  return e;
}

void make_up_roots(int W, int U, float2* out) {
  const double pi = 3.14159265358979323846;
  const int n = U * W;
  for (int m = 0; m < n; ++m) {
    const double th = 2.0 * pi * (double)m / (double)n;
    out[m] = make_float2((float)std::cos(th), (float)std::sin(th));
  }
}

cudaError_t launch_xcorr_cols(const RefGeo& g, float2* scratch, int npl, int M, int npatch,
                              const float2* tw, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(g.W, {
    using G = Line<WW>;
    e = launch_pdl(k_xcorr_cols<WW>, dim3(WW / g.CBX, npatch), dim3(g.CBX * G::L), g.smX, s,
                   scratch, npl, M, g.CBX, tw);
  });
  return e;
}

cudaError_t launch_xcorrb_rows(const RefGeo& g, float2* scratch, int npl, int plane,
                               int nplanes, int npatch, const float2* tw, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(g.W, {
    using G = Line<WW>;
    const int thr = (g.RX * G::L + 31) / 32 * 32;
    e = launch_pdl(k_xcorrb_rows<WW>, dim3(nplanes * WW / g.RX, npatch), dim3(thr), g.smR, s,
                   scratch, npl, plane, g.RX, tw);
  });
  return e;
}

cudaError_t launch_xcorr_rows(const RefGeo& g, const float2* scratch, int npl, int M,
                              int npatch, const float2* tw, float* cval, int* cidx,
                              cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(g.W, {
    using G = Line<WW>;
    const int thr = (g.RX * G::L + 31) / 32 * 32;
    e = launch_pdl(k_xcorr_rows<WW>, dim3(WW / g.RX, npatch), dim3(thr), g.smR, s, scratch, npl,
                   M, g.RX, tw, cval, cidx);
  });
  return e;
}

cudaError_t launch_updft(const RefGeo& g, float2* scratch, int npl, int M, const int* ids,
                         int npatch, const float* cval, const int* cidx, const float2* roots,
                         float2* part, float* shift, float* gap, int* done, int* err,
                         cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  const int nparts = g.W / g.RX;
  if (g.U <= 1) {
    k_coarse_only<<<npatch, 128, 0, s>>>(ids, nparts, g.W, cval, cidx, shift, gap);
    return cudaGetLastError();
  }
  const int nblocks = g.tc ? (g.W + kTcRows - 1) / kTcRows : g.W / g.RB;
  cudaError_t e = cudaSuccess;
  if (g.tc) {  // the shares are added by the last CTA of each patch
    const size_t sm = (size_t)kTcFixed;
    PTY_DISPATCH_W(g.W, e = launch_pdl(k_updft_tc<WW>, dim3(nblocks, npatch), dim3(256), sm, s,
                                       scratch, npl, M, nparts, cval, cidx, roots, g.U, g.K,
                                       part, ids, done, shift, gap, err));
    return e;
  } else {
    PTY_DISPATCH_W(g.W, e = launch_pdl(k_updft_part<WW>, dim3(nblocks, npatch), dim3(512), g.smU,
                                       s, scratch, npl, M, nparts, cval, cidx, roots, g.U, g.K,
                                       g.RB, part));
  }
  if (e != cudaSuccess) return e;
  return launch_pdl(k_updft_final, dim3(npatch), dim3(256), 0, s, ids, g.W, nblocks, nparts,
                    cval, cidx, g.U, g.K, part, shift, gap);
}

cudaError_t launch_adam(float* pos, float* m, float* v, const float* g, int N, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, float max_step,
                        float ymax, float xmax, cudaStream_t s) {
  const int n = 2 * N;
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(pos, m, v, g, N, lr, b1, b2, eps, bc1, bc2, max_step,
                                         ymax, xmax);
  return cudaGetLastError();
}

}  // namespace pty
