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
  // both columns are requested together
  float2 v[G::N1], vb[G::N1];
  if (act && lane < G::N2) {
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) {
      v[n1] = colA[(size_t)(G::N2 * n1 + lane) * W];
      vb[n1] = colB[(size_t)(G::N2 * n1 + lane) * W];
    }
  }
  __syncthreads();
  // A = F(o_j): the column DFTs of plane M (its row DFTs come from pass A)
  if (act && lane < G::N2) fwd_step1<W>(v, lane, tw, lbuf);
  __syncthreads();
  float2 za[G::N2];
  if (act && lane < G::N1) fwd_step3<W>(za, lane, lbuf);
  __syncthreads();
  // B = F(o'_j)
  if (act && lane < G::N2) fwd_step1<W>(vb, lane, tw, lbuf);
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
// XCORR_B: forward row DFTs of the two real images pass B left in planes M
// (model intensity) and M + 1 (counts); the correlation passes then take
// them exactly as they take the two crops' row DFTs for XCORR_A.  The two
// planes are consecutive, so a CTA's RX lines are rows of a 2W-row block.
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
  pdl_wait();  // both images come from the column pass
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

__global__ void __launch_bounds__(256)
k_updft_final(const int* __restrict__ ids, int W, int nblocks, int nparts,
              const float* __restrict__ cval, const int* __restrict__ cidx, int U, int K,
              const float2* __restrict__ part, float* __restrict__ shift,
              float* __restrict__ gap) {
  __shared__ float rv[32];
  __shared__ int ri[32];
  pdl_trigger();
  pdl_wait();  // the partial sums come from updft_part
  const int lp = blockIdx.x, j = ids[lp];
  int sy, sx;
  coarse_peak(cval, cidx, lp, nparts, W, sy, sx, rv, ri);
  const int half = K / 2;
  float best = -1.f, second = -1.f;
  int bi = 0x7fffffff;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < nblocks; ++b)
      acc = cadd(acc, part[((size_t)lp * nblocks + b) * K * K + e]);  // fixed order
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

RefGeo make_refgeo(int W, int U) {
  RefGeo g{};
  g.W = W;
  g.U = std::max(1, U);
  g.K = (int)std::ceil(1.5 * g.U);
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

cudaError_t launch_xcorrb_rows(const RefGeo& g, float2* scratch, int npl, int M, int npatch,
                               const float2* tw, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(g.W, {
    using G = Line<WW>;
    const int thr = (g.RX * G::L + 31) / 32 * 32;
    e = launch_pdl(k_xcorrb_rows<WW>, dim3(2 * WW / g.RX, npatch), dim3(thr), g.smR, s, scratch,
                   npl, M, g.RX, tw);
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
                         float2* part, float* shift, float* gap, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  const int nparts = g.W / g.RX;
  if (g.U <= 1) {
    k_coarse_only<<<npatch, 128, 0, s>>>(ids, nparts, g.W, cval, cidx, shift, gap);
    return cudaGetLastError();
  }
  const int nblocks = g.W / g.RB;
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(g.W, e = launch_pdl(k_updft_part<WW>, dim3(nblocks, npatch), dim3(512), g.smU,
                                     s, scratch, npl, M, nparts, cval, cidx, roots, g.U, g.K,
                                     g.RB, part));
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
