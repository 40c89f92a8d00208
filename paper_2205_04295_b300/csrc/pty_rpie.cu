// M-rPIE group step on sm_103a: the three passes over one chunk of a group of
// pairwise-disjoint crop boxes, the probe update at the end of the group, and
// small reductions.  Equations are those of the M-rPIE section of Guzzi et
// al. (arXiv 2205.04295): exit waves (Eq. 1, per mode as in Eq. 4), far-field
// propagation (Eq. 2, unitary DFT), the mixed-state modulus constraint
// (Eq. 7), the object update (Eq. 6) and the probe update (Eq. 5).
//
// Pass A  rows_fwd : per (row block, patches): psi_p = P_p o_j for every mode,
//                    forward row DFTs, rows written to the far-field scratch;
//                    also the row block's max |o_j|^2.
// Pass B  cols     : per (column block, patch): forward column DFTs of every
//                    mode, S = sum_p |Psi_p|^2, Psi'_p = sqrt(I)/(sqrt(S)+eps)
//                    Psi_p, error partial sum, inverse column DFTs.
// Pass C  rows_inv : per (row block, patches): inverse row DFTs -> psi'_p,
//                    D_p = psi'_p - psi_p, object update written in place
//                    (boxes of a group are disjoint), probe numerator /
//                    denominator partial sums kept per CTA column.
// probe_apply      : P_p += alpha_P sum(num_p) / sum(den), fixed-order sums
//                    over the CTA-column partials; new max_r sum_p |P_p|^2.
//
// All reductions run in a fixed order, so results are bitwise repeatable.
#include "pty_fft.cuh"
#include "pty_internal.h"

#include <algorithm>
#include <cmath>

namespace pty {

namespace {

PTY_D float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
PTY_D float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Block-wide reductions; every thread gets the result.  Contain barriers.
PTY_D float block_sum(float v, float* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < nw; ++i) t += red[i];  // fixed order
  return t;
}
PTY_D float block_max(float v, float* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < nw; ++i) t = fmaxf(t, red[i]);
  return t;
}

// ---------------------------------------------------------------- pass A
template <int W>
PTY_D void rows_fwd_body(const float2* O, int Hx, const float2* P,
           int M, int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           const float2* __restrict__ tw_g, float2* __restrict__ scratch,
           float* __restrict__ omax_part, int npl, int xo, int bx, int by) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* Prow = tw + W;
  float2* tbuf = Prow + M * R * W;
  __shared__ float red[32];

  const int r0 = bx * R;
  const int nrb = W / R;
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) {
    const int k = e / (R * W), rem = e - k * R * W, r = rem / W, c = rem - r * W;
    Prow[e] = P[((size_t)k * W + r0 + r) * W + c];
  }
  __syncthreads();

  // lines: (mode k, row r) for k < M, and with xo the crop itself as plane M
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < (M + xo) * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  const int p0 = by * ppc, p1 = min(npatch, p0 + ppc);
  // crop rows of patch lp + 1 are loaded while patch lp is transformed
  float2 on[G::N1];
  if (p0 < p1 && act && lane < G::N2) {
    const int2 cc = corners[ids[p0]];
    const float2* orow = O + (size_t)(cc.x + r0 + r) * Hx + cc.y;
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) on[n1] = orow[G::N2 * n1 + lane];
  }
  for (int lp = p0; lp < p1; ++lp) {
    float omax = 0.f;
    if (act && lane < G::N2) {
      const float2* prow = Prow + (k * R + r) * W;
      float2 v[G::N1];
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) {
        const int c = G::N2 * n1 + lane;
        const float2 o = on[n1];
        v[n1] = k < M ? cmul(prow[c], o) : o;
        omax = fmaxf(omax, cabs2(o));
      }
      if (lp + 1 < p1) {
        const int2 cn = corners[ids[lp + 1]];
        const float2* orow = O + (size_t)(cn.x + r0 + r) * Hx + cn.y;
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) on[n1] = orow[G::N2 * n1 + lane];
      }
      fwd_step1<W>(v, lane, tw, lbuf);
    }
    __syncthreads();
    if (act && lane < G::N1) {
      float2 z[G::N2];
      fwd_step3<W>(z, lane, lbuf);
      float2* dst = scratch + (((size_t)lp * npl + k) * W + r0 + r) * W;
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = z[k2];
    }
    omax = block_max(omax, red);  // its barriers also guard lbuf reuse
    if (threadIdx.x == 0) omax_part[(size_t)lp * nrb + bx] = omax;
  }
}

template <int W>
__global__ void __launch_bounds__(256)
k_rows_fwd(const float2* __restrict__ O, int Hx, const float2* __restrict__ P,
           int M, int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           const float2* __restrict__ tw_g, float2* __restrict__ scratch,
           float* __restrict__ omax_part, int npl, int xo) {
  rows_fwd_body<W>(O, Hx, P, M, R, ppc, ids, corners, npatch, tw_g, scratch, omax_part, npl, xo, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- pass B
// GRAD = false: the modulus constraint (Eq. 7).  GRAD = true: the Fourier-
// domain step of the amplitude-loss adjoint, G_Psi = 2 (1 - sqrt(I) / A) Psi
// with A = sqrt(S + eps) (eps carries delta), and the loss partial sums.
template <int W, bool GRAD>
PTY_D void cols_body(float2* __restrict__ scratch, int M, int CB,
       const uint16_t* __restrict__ I, const int* __restrict__ ids,
       const float2* __restrict__ tw_g, float inv_w, float eps,
       float* __restrict__ err_part, int npl, int xo, int ppcb, int npatch, int bx, int by) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  float* Sb = reinterpret_cast<float*>(tbuf + (M + xo) * CB * G::LP);
  float* Isq = Sb + M * CB * W;  // sqrt of the counts of this column block
  __shared__ float red[32];

  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  const int c0 = bx * CB;
  const int c = threadIdx.x % CB, rest = threadIdx.x / CB;
  const int lane = rest % G::L, k = rest / G::L;
  // k < M: the modes; k == M (with xo): the crop, forward transform only
  const bool act = k < M + xo;
  const bool mode = k < M;
  float2* lbuf = tbuf + ((act ? k : 0) * CB + c) * G::LP;
  const int p0 = by * ppcb, p1 = min(npatch, p0 + ppcb);
  __syncthreads();
  for (int lp = p0; lp < p1; ++lp) {
    const int j = ids[lp];
    float2* col = scratch + ((size_t)lp * npl + (act ? k : 0)) * W * W + c0 + c;
    float2 v[G::N1];
    if (act && lane < G::N2) {
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = col[(size_t)(G::N2 * n1 + lane) * W];
    }
    {
      // the counts are requested together with the columns: one round trip
      const uint16_t* Ij = I + (size_t)j * W * W;
      for (int el = threadIdx.x; el < CB * W; el += blockDim.x) {
        const int u = el / CB, cl = el - u * CB;
        Isq[el] = sqrtf((float)__ldcs(Ij + (size_t)((u + W / 2) % W) * W + (c0 + cl + W / 2) % W));
      }
    }
    if (act && lane < G::N2) fwd_step1<W>(v, lane, tw, lbuf);
    __syncthreads();
    float2 z[G::N2];
    if (act && lane < G::N1) {
      fwd_step3<W>(z, lane, lbuf);
      if (mode) {
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2)
          Sb[(k * W + lane + G::N1 * k2) * CB + c] = cabs2(z[k2]);
      } else {
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) col[(size_t)(lane + G::N1 * k2) * W] = z[k2];
      }
    }
    __syncthreads();
    // constraint factor once per detector pixel (u, c): S = sum_k |Psi_k|^2 in a
    // fixed mode order, f = sqrt(I) / (sqrt(S) + eps) folded with both 1/W
    // normalisations; stored over mode 0's |Psi|^2.
    float e = 0.f;
    {
      const float f2 = inv_w * inv_w;
      for (int el = threadIdx.x; el < CB * W; el += blockDim.x) {
        const int u = el / CB, cl = el - u * CB;
        float s = 0.f;
        for (int kk = 0; kk < M; ++kk) s += Sb[(kk * W + u) * CB + cl];
        const float sI = Isq[el];
        if (!GRAD) {
          const float a = sqrtf(s) * inv_w;
          const float d = a - sI;
          e = fmaf(d, d, e);
          Sb[u * CB + cl] = sI / (a + eps) * f2;
        } else {
          const float a = sqrtf(fmaf(s, f2, eps));
          const float d = a - sI;
          e = fmaf(d, d, e);
          Sb[u * CB + cl] = 2.f * (1.f - sI / a) * f2;
        }
      }
    }
    __syncthreads();
    if (mode && lane < G::N1) {
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2)
        z[k2] = cscale(z[k2], Sb[(lane + G::N1 * k2) * CB + c]);
      inv_stepA<W>(z, lane, tw, lbuf);
    }
    __syncthreads();
    if (mode && lane < G::N2) {
      inv_stepB<W>(v, lane, lbuf);
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) col[(size_t)(G::N2 * n1 + lane) * W] = v[n1];
    }
    e = block_sum(e, red);  // its barriers also guard lbuf and Sb reuse
    if (threadIdx.x == 0) err_part[(size_t)j * (W / CB) + bx] = e;
  }
}


template <int W, bool GRAD>
__global__ void __launch_bounds__(384)
k_cols(float2* __restrict__ scratch, int M, int CB,
       const uint16_t* __restrict__ I, const int* __restrict__ ids,
       const float2* __restrict__ tw_g, float inv_w, float eps,
       float* __restrict__ err_part, int npl, int xo, int ppcb, int npatch) {
  cols_body<W, GRAD>(scratch, M, CB, I, ids, tw_g, inv_w, eps, err_part, npl, xo, ppcb, npatch,
                     blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- pass C
template <int W>
PTY_D void rows_inv_body(float2* O, int Hx, const float2* P, int M,
           int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           float2* scratch, const float* omax_part,
           const float* pmax_part, int n_pmax,
           const float2* __restrict__ tw_g, UpdArgs a,
           float2* pnum, float* pden,
           float* osum, int accumulate, int npl, int refine, int bx, int by) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  const int TB = max(M * R * G::LP, M * R * W);
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* Prow = tw + W;
  float2* tbuf = Prow + M * R * W;  // transpose buffer, then D conj(P) terms
  float2* num = tbuf + TB;
  float2* ostash = num + M * R * W;  // the crop rows of the current patch
  float2* onew = ostash + R * W;     // refined crop rows (refine only)
  float* invd = reinterpret_cast<float*>(onew + (refine ? R * W : 0));  // alpha_O / denominator
  float* den = invd + R * W;
  __shared__ float s_pmax, s_omax;

  const int r0 = bx * R;
  const int nrb = W / R;
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) {
    const int k = e / (R * W), rem = e - k * R * W, r = rem / W, c = rem - r * W;
    Prow[e] = P[((size_t)k * W + r0 + r) * W + c];
    num[e] = make_float2(0.f, 0.f);
  }
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int i = threadIdx.x; i < n_pmax; i += 32) m = fmaxf(m, pmax_part[i]);
    m = warp_max(m);
    if (threadIdx.x == 0) s_pmax = m;
  }
  __syncthreads();
  {
    const float pmax = s_pmax;
    const float gden = a.gamma * pmax + a.reg_eps * pmax;
    for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
      float s = 0.f;
      for (int k = 0; k < M; ++k) s += cabs2(Prow[k * R * W + e]);
      const float dn = fmaf(1.f - a.gamma, s, gden);
      invd[e] = dn > 0.f ? a.alpha_O / dn : 0.f;  // a zero denominator has a zero numerator
      den[e] = 0.f;
    }
  }

  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < M * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  const int p0 = by * ppc, p1 = min(npatch, p0 + ppc);
  float osum_local = 0.f;
  for (int lp = p0; lp < p1; ++lp) {
    const int2 cc = corners[ids[lp]];
    // the far-field rows and the crop rows are requested together: one
    // global round trip per patch
    float2 z[G::N2];
    if (act && lane < G::N1) {
      const float2* src = scratch + (((size_t)lp * npl + k) * W + r0 + r) * W;
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = src[lane + G::N1 * k2];
    }
    if (act && k == 0 && lane < G::N2) {
      const float2* orow = O + (size_t)(cc.x + r0 + r) * Hx + cc.y;
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) ostash[r * W + G::N2 * n1 + lane] = orow[G::N2 * n1 + lane];
    }
    if (threadIdx.x < 32) {
      float m = 0.f;
      for (int i = threadIdx.x; i < nrb; i += 32) m = fmaxf(m, omax_part[(size_t)lp * nrb + i]);
      m = warp_max(m);
      if (threadIdx.x == 0) s_omax = m;
    }
    if (act && lane < G::N1) inv_stepA<W>(z, lane, tw, lbuf);
    __syncthreads();
    float2 v[G::N1];
    if (act && lane < G::N2) inv_stepB<W>(v, lane, lbuf);
    __syncthreads();  // tbuf is reused below for the D conj(P) terms
    if (act && lane < G::N2) {
      float2* T = tbuf + (k * R + r) * W;
      float2* nm = num + (k * R + r) * W;
      const float2* prow = Prow + (k * R + r) * W;
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) {
        const int c = G::N2 * n1 + lane;
        const float2 o = ostash[r * W + c];
        const float2 Pk = prow[c];
        const float2 D = csub(v[n1], cmul(Pk, o));
        T[c] = cmulc(D, Pk);
        nm[c] = cadd(nm[c], cmulc(D, o));
      }
    }
    __syncthreads();
    const float om = s_omax;
    for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
      const int rr = e / W, c = e - rr * W;
      const float2 o = ostash[e];
      float2 s = make_float2(0.f, 0.f);
      for (int kk = 0; kk < M; ++kk) s = cadd(s, tbuf[(kk * R + rr) * W + c]);
      const float sc = invd[e];
      const float2 onw = make_float2(fmaf(sc, s.x, o.x), fmaf(sc, s.y, o.y));
      O[(size_t)(cc.x + r0 + rr) * Hx + cc.y + c] = onw;
      if (refine) onew[e] = onw;
      den[e] += fmaf(1.f - a.beta, cabs2(o), a.beta * om);
    }
    osum_local += om;
    __syncthreads();
    if (refine) {
      // forward row DFTs of the refined crop o'_j -> plane M + 1 (XCORR_A)
      if (line < R && lane < G::N2) {
        float2 v2[G::N1];
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) v2[n1] = onew[line * W + G::N2 * n1 + lane];
        fwd_step1<W>(v2, lane, tw, tbuf + line * G::LP);
      }
      __syncthreads();
      if (line < R && lane < G::N1) {
        float2 zz[G::N2];
        fwd_step3<W>(zz, lane, tbuf + line * G::LP);
        float2* dst = scratch + (((size_t)lp * npl + M + 1) * W + r0 + line) * W;
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = zz[k2];
      }
      __syncthreads();
    }
  }
  const int slot = by;
  for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) {
    const int kk = e / (R * W), rem = e - kk * R * W, rr = rem / W, c = rem - rr * W;
    const size_t g = (((size_t)slot * M + kk) * W + r0 + rr) * W + c;
    pnum[g] = accumulate ? cadd(pnum[g], num[e]) : num[e];
  }
  for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
    const int rr = e / W, c = e - rr * W;
    const size_t g = ((size_t)slot * W + r0 + rr) * W + c;
    pden[g] = accumulate ? pden[g] + den[e] : den[e];
  }
  if (bx == 0 && threadIdx.x == 0)
    osum[slot] = accumulate ? osum[slot] + osum_local : osum_local;
}

template <int W>
__global__ void __launch_bounds__(256, 2)
k_rows_inv(float2* __restrict__ O, int Hx, const float2* __restrict__ P, int M,
           int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           float2* __restrict__ scratch, const float* __restrict__ omax_part,
           const float* __restrict__ pmax_part, int n_pmax,
           const float2* __restrict__ tw_g, UpdArgs a,
           float2* __restrict__ pnum, float* __restrict__ pden,
           float* __restrict__ osum, int accumulate, int npl, int refine) {
  rows_inv_body<W>(O, Hx, P, M, R, ppc, ids, corners, npatch, scratch, omax_part, pmax_part, n_pmax, tw_g, a, pnum, pden, osum, accumulate, npl, refine, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------- probe apply
PTY_D void probe_apply_body(float2* P, int M, int WW, const float2* pnum, const float* pden,
                            const float* osum, int nslots, float alpha_P, float reg_eps,
                            float* pmax_part, int bx, int gx) {
  __shared__ float red[32];
  float os = 0.f;
  for (int s = 0; s < nslots; ++s) os += osum[s];
  const float guard = reg_eps * os;
  float lmax = 0.f;
  for (int pix = bx * blockDim.x + threadIdx.x; pix < WW; pix += gx * blockDim.x) {
    float d = 0.f;
    for (int s = 0; s < nslots; ++s) d += pden[(size_t)s * WW + pix];
    const float dd = d + guard;
    const float sc = dd > 0.f ? alpha_P / dd : 0.f;  // zero numerator too
    float pint = 0.f;
    for (int k = 0; k < M; ++k) {
      float2 n = make_float2(0.f, 0.f);
      for (int s = 0; s < nslots; ++s) n = cadd(n, pnum[((size_t)s * M + k) * WW + pix]);
      float2 p = P[(size_t)k * WW + pix];
      p = make_float2(fmaf(sc, n.x, p.x), fmaf(sc, n.y, p.y));
      P[(size_t)k * WW + pix] = p;
      pint += cabs2(p);
    }
    lmax = fmaxf(lmax, pint);
  }
  lmax = block_max(lmax, red);
  if (threadIdx.x == 0) pmax_part[bx] = lmax;
}

__global__ void __launch_bounds__(256)
k_probe_apply(float2* __restrict__ P, int M, int WW, const float2* __restrict__ pnum,
              const float* __restrict__ pden, const float* __restrict__ osum,
              int nslots, float alpha_P, float reg_eps, float* __restrict__ pmax_part) {
  probe_apply_body(P, M, WW, pnum, pden, osum, nslots, alpha_P, reg_eps, pmax_part, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256)
k_pmax(const float2* __restrict__ P, int M, int WW, float* __restrict__ pmax_part) {
  __shared__ float red[32];
  float lmax = 0.f;
  for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < WW; pix += gridDim.x * blockDim.x) {
    float pint = 0.f;
    for (int k = 0; k < M; ++k) pint += cabs2(P[(size_t)k * WW + pix]);
    lmax = fmaxf(lmax, pint);
  }
  lmax = block_max(lmax, red);
  if (threadIdx.x == 0) pmax_part[blockIdx.x] = lmax;
}

PTY_D void err_reduce_body(const float* part, size_t n, double inv_sumI, float* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)(red[0] * inv_sumI);
}

__global__ void __launch_bounds__(1024)
k_err_reduce(const float* __restrict__ part, size_t n, double inv_sumI, float* out) {
  err_reduce_body(part, n, inv_sumI, out);
}

// Model intensities: forward column DFTs after pass A, S written out.
template <int W>
__global__ void __launch_bounds__(512)
k_cols_intensity(const float2* __restrict__ scratch, int M, int CB,
                 const int* __restrict__ ids, const float2* __restrict__ tw_g,
                 float inv_w, float* __restrict__ out) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  float* Sb = reinterpret_cast<float*>(tbuf + M * CB * G::LP);
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  const int lp = blockIdx.y, c0 = blockIdx.x * CB;
  const int c = threadIdx.x % CB, rest = threadIdx.x / CB;
  const int lane = rest % G::L, k = rest / G::L;
  const bool act = k < M;
  const int j = ids[lp];
  const float2* col = scratch + ((size_t)lp * M + (act ? k : 0)) * W * W + c0 + c;
  float2* lbuf = tbuf + ((act ? k : 0) * CB + c) * G::LP;
  __syncthreads();
  if (act && lane < G::N2) {
    float2 v[G::N1];
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = col[(size_t)(G::N2 * n1 + lane) * W];
    fwd_step1<W>(v, lane, tw, lbuf);
  }
  __syncthreads();
  if (act && lane < G::N1) {
    float2 z[G::N2];
    fwd_step3<W>(z, lane, lbuf);
#pragma unroll
    for (int k2 = 0; k2 < G::N2; ++k2)
      Sb[(k * CB + c) * W + lane + G::N1 * k2] = cabs2(z[k2]);
  }
  __syncthreads();
  const float f2 = inv_w * inv_w;
  for (int e = threadIdx.x; e < CB * W; e += blockDim.x) {
    const int u = e / CB, cl = e - u * CB;
    float s = 0.f;
    for (int kk = 0; kk < M; ++kk) s += Sb[(kk * CB + cl) * W + u];
    const int iu = (u + W / 2) % W, iv = (c0 + cl + W / 2) % W;
    out[((size_t)j * W + iu) * W + iv] = s * f2;
  }
}

// Plain batched 2-D DFT through the same line steps (rows, then columns).
template <int W, bool INV>
__global__ void __launch_bounds__(256) k_fft_rows(float2* __restrict__ data, int nrows) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  const int lines = blockDim.x / G::L;
  for (int e = threadIdx.x; e < W; e += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * e / W, &sn, &cs);
    tw[e] = make_float2((float)cs, (float)sn);
  }
  __syncthreads();
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const int row = blockIdx.x * lines + line;
  const bool act = line < lines && row < nrows;
  float2* x = data + (size_t)(act ? row : 0) * W;
  float2* lbuf = tbuf + line * G::LP;
  if (!INV) {
    if (act && lane < G::N2) {
      float2 v[G::N1];
      for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = x[G::N2 * n1 + lane];
      fwd_step1<W>(v, lane, tw, lbuf);
    }
    __syncthreads();
    if (act && lane < G::N1) {
      float2 z[G::N2];
      fwd_step3<W>(z, lane, lbuf);
      for (int k2 = 0; k2 < G::N2; ++k2) x[lane + G::N1 * k2] = z[k2];
    }
  } else {
    if (act && lane < G::N1) {
      float2 z[G::N2];
      for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = x[lane + G::N1 * k2];
      inv_stepA<W>(z, lane, tw, lbuf);
    }
    __syncthreads();
    if (act && lane < G::N2) {
      float2 v[G::N1];
      inv_stepB<W>(v, lane, lbuf);
      for (int n1 = 0; n1 < G::N1; ++n1) x[G::N2 * n1 + lane] = v[n1];
    }
  }
}

template <int W, bool INV>
__global__ void __launch_bounds__(256) k_fft_cols(float2* __restrict__ data, int CB) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  for (int e = threadIdx.x; e < W; e += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * e / W, &sn, &cs);
    tw[e] = make_float2((float)cs, (float)sn);
  }
  __syncthreads();
  const int c = threadIdx.x % CB, lane = threadIdx.x / CB;  // lanes >= L stay idle
  float2* col = data + (size_t)blockIdx.y * W * W + blockIdx.x * CB + c;
  float2* lbuf = tbuf + c * G::LP;
  if (!INV) {
    if (lane < G::N2) {
      float2 v[G::N1];
      for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = col[(size_t)(G::N2 * n1 + lane) * W];
      fwd_step1<W>(v, lane, tw, lbuf);
    }
    __syncthreads();
    if (lane < G::N1) {
      float2 z[G::N2];
      fwd_step3<W>(z, lane, lbuf);
      for (int k2 = 0; k2 < G::N2; ++k2) col[(size_t)(lane + G::N1 * k2) * W] = z[k2];
    }
  } else {
    if (lane < G::N1) {
      float2 z[G::N2];
      for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = col[(size_t)(lane + G::N1 * k2) * W];
      inv_stepA<W>(z, lane, tw, lbuf);
    }
    __syncthreads();
    if (lane < G::N2) {
      float2 v[G::N1];
      inv_stepB<W>(v, lane, lbuf);
      for (int n1 = 0; n1 < G::N1; ++n1) col[(size_t)(G::N2 * n1 + lane) * W] = v[n1];
    }
  }
}

__global__ void k_finite(const float* __restrict__ p, size_t n, int* flag) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(p[i])) {
      *flag = 1;
      return;
    }
}

int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}
int round32(int v) { return (v + 31) / 32 * 32; }

template <int W> void geo(int& L, int& LP) {
  L = Line<W>::L;
  LP = Line<W>::LP;
}

}  // namespace

int smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 227 * 1024;
  }
  return v;
}

cudaError_t allow_max_smem(const void* func) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin() - (int)fa.sharedSizeBytes);
}

int lanes_per_line(int W) {
  int L = 16, LP = 0;
  switch (W) {
    case 32: geo<32>(L, LP); break;
    case 64: geo<64>(L, LP); break;
    case 96: geo<96>(L, LP); break;
    case 128: geo<128>(L, LP); break;
    case 192: geo<192>(L, LP); break;
    default: geo<256>(L, LP); break;
  }
  return L;
}

bool supported_W(int W) {
  return W == 32 || W == 64 || W == 96 || W == 128 || W == 192 || W == 256;
}

#define PTY_DISPATCH_W(W, ...)                               \
  switch (W) {                                               \
    case 32: { constexpr int WW = 32; __VA_ARGS__; } break;   \
    case 64: { constexpr int WW = 64; __VA_ARGS__; } break;   \
    case 96: { constexpr int WW = 96; __VA_ARGS__; } break;   \
    case 128: { constexpr int WW = 128; __VA_ARGS__; } break; \
    case 192: { constexpr int WW = 192; __VA_ARGS__; } break; \
    case 256: { constexpr int WW = 256; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;                   \
  }

Tiling make_tiling(int W, int M, bool refine, int max_threads_b_req, int R_req, int ppc_req,
                   int CB_req) {
  Tiling t{};
  t.W = W;
  t.M = M;
  t.xo = refine ? 1 : 0;
  t.refine = refine ? 1 : 0;
  t.npl = refine ? M + 2 : M;
  int L = 16, LP = W;
  switch (W) {
    case 32: geo<32>(L, LP); break;
    case 64: geo<64>(L, LP); break;
    case 96: geo<96>(L, LP); break;
    case 128: geo<128>(L, LP); break;
    case 192: geo<192>(L, LP); break;
    default: geo<256>(L, LP); break;
  }
  const int MA = M + t.xo;  // lines per row in pass A, columns-groups in pass B
  const int max_threads_b = std::min(max_threads_b_req, 384);
  int R = pow2_floor(std::max(1, 256 / (MA * L)));
  R = std::min(R, 16);
  while (W % R) R /= 2;
  if (R_req > 0) R = R_req;
  t.R = R;
  t.ppc = ppc_req > 0 ? ppc_req : 4;
  t.ppcb = 2;
  int CB = pow2_floor(std::max(1, max_threads_b / (MA * L)));
  CB = std::max(2, std::min(16, CB));  // MA * CB * L <= max_threads_b threads
  while ((W / 2) % CB) CB /= 2;
  if (CB_req > 0) CB = CB_req;
  t.CB = CB;
  t.thrA = round32(MA * R * L);
  t.thrC = round32(M * R * L);
  t.thrB = round32(MA * CB * L);
  t.smA = (size_t)(W + M * R * W + MA * R * LP) * sizeof(float2);
  t.smB = (size_t)(W + MA * CB * LP) * sizeof(float2) + (size_t)(M + 1) * CB * W * sizeof(float);
  t.smI = (size_t)(W + M * CB * LP) * sizeof(float2) + (size_t)M * CB * W * sizeof(float);
  const int TB = std::max(M * R * LP, M * R * W);
  t.smC = (size_t)(W + M * R * W + TB + M * R * W + R * W + (refine ? R * W : 0)) * sizeof(float2) +
          (size_t)2 * R * W * sizeof(float);
  t.n_pmax = std::max(1, std::min(1024, W * W / 256));
  return t;
}

cudaError_t set_smem_limits(const Tiling& t) {
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(t.W, {
    e = allow_max_smem((const void*)k_rows_fwd<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_cols<WW, false>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_cols<WW, true>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_rows_inv<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_cols_intensity<WW>);
  });
  return e;
}

void make_twiddles(int W, float2* out) {
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < W; ++m) {
    const double th = -2.0 * pi * (double)m / (double)W;
    out[m] = make_float2((float)std::cos(th), (float)std::sin(th));
  }
}

cudaError_t launch_rows_fwd(const Tiling& t, const float2* O, int Hx, const float2* P,
                            const int* ids, const int2* corners, int npatch,
                            const float2* tw, float2* scratch, float* omax_part,
                            cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppc - 1) / t.ppc);
  PTY_DISPATCH_W(t.W, (k_rows_fwd<WW><<<grid, t.thrA, t.smA, s>>>(O, Hx, P,
                                    t.M, t.R, t.ppc, ids, corners, npatch, tw, scratch,
                                    omax_part, t.npl, t.xo)));
  return cudaGetLastError();
}

// Pass A with the plain layout (M planes, no crop plane) whatever t says:
// used by the model-intensity computation.
cudaError_t launch_rows_fwd_plain(const Tiling& t, const float2* O, int Hx, const float2* P,
                                  const int* ids, const int2* corners, int npatch,
                                  const float2* tw, float2* scratch, float* omax_part,
                                  cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppc - 1) / t.ppc);
  PTY_DISPATCH_W(t.W, (k_rows_fwd<WW><<<grid, t.thrA, t.smA, s>>>(
                          O, Hx, P, t.M, t.R, t.ppc, ids, corners, npatch, tw,
                          scratch, omax_part, t.M, 0)));
  return cudaGetLastError();
}

cudaError_t launch_cols(const Tiling& t, float2* scratch, const uint16_t* I,
                        const int* ids, int npatch, const float2* tw, float inv_w,
                        float eps, float* err_part, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.CB, (npatch + t.ppcb - 1) / t.ppcb);
  PTY_DISPATCH_W(t.W, (k_cols<WW, false><<<grid, t.thrB, t.smB, s>>>(scratch,
                                    t.M, t.CB, I, ids, tw, inv_w, eps, err_part, t.npl, t.xo,
                                    t.ppcb, npatch)));
  return cudaGetLastError();
}

cudaError_t launch_cols_grad(const Tiling& t, float2* scratch, const uint16_t* I,
                             const int* ids, int npatch, const float2* tw, float inv_w,
                             float delta, float* loss_part, int npl, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.CB, (npatch + t.ppcb - 1) / t.ppcb);
  PTY_DISPATCH_W(t.W, (k_cols<WW, true><<<grid, t.thrB, t.smB, s>>>(
                          scratch, t.M, t.CB, I, ids, tw, inv_w, delta, loss_part, npl, 0,
                          t.ppcb, npatch)));
  return cudaGetLastError();
}

cudaError_t launch_rows_inv(const Tiling& t, float2* O, int Hx, const float2* P,
                            const int* ids, const int2* corners, int npatch,
                            float2* scratch, const float* omax_part,
                            const float* pmax_part, const float2* tw,
                            const UpdArgs& a, float2* pnum, float* pden,
                            float* osum, int accumulate, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppc - 1) / t.ppc);
  PTY_DISPATCH_W(t.W, (k_rows_inv<WW><<<grid, t.thrC, t.smC, s>>>(O, Hx, P,
                                    t.M, t.R, t.ppc, ids, corners, npatch, scratch, omax_part,
                                    pmax_part, t.n_pmax, tw, a, pnum, pden, osum, accumulate,
                                    t.npl, t.refine)));
  return cudaGetLastError();
}

cudaError_t launch_probe_apply(const Tiling& t, float2* P, const float2* pnum,
                               const float* pden, const float* osum, int nslots,
                               float alpha_P, float reg_eps, float* pmax_part,
                               cudaStream_t s) {
  k_probe_apply<<<t.n_pmax, 256, 0, s>>>(P, t.M, t.W * t.W, pnum, pden, osum, nslots,
                                         alpha_P, reg_eps, pmax_part);
  return cudaGetLastError();
}

cudaError_t launch_pmax(const Tiling& t, const float2* P, float* pmax_part, cudaStream_t s) {
  k_pmax<<<t.n_pmax, 256, 0, s>>>(P, t.M, t.W * t.W, pmax_part);
  return cudaGetLastError();
}

cudaError_t launch_err_reduce(const float* err_part, size_t n, double inv_sumI, float* out,
                              cudaStream_t s) {
  k_err_reduce<<<1, 1024, 0, s>>>(err_part, n, inv_sumI, out);
  return cudaGetLastError();
}

cudaError_t launch_cols_intensity(const Tiling& t, const float2* scratch, const int* ids,
                                  int npatch, const float2* tw, float inv_w, float* out,
                                  cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.CB, npatch);
  PTY_DISPATCH_W(t.W, (k_cols_intensity<WW><<<grid, t.thrB, t.smI, s>>>(
                          scratch, t.M, t.CB, ids, tw, inv_w, out)));
  return cudaGetLastError();
}

cudaError_t launch_fft2(void* data, int W, int batch, int inverse, const float2*,
                        cudaStream_t s) {
  float2* d = static_cast<float2*>(data);
  const int nrows = W * batch;
  PTY_DISPATCH_W(W, {
    using G = Line<WW>;
    const int lines = 256 / G::L;
    const dim3 gr((nrows + lines - 1) / lines);
    const size_t smr = (size_t)(WW + lines * G::LP) * sizeof(float2);
    const int CB = pow2_floor(256 / G::L);
    const dim3 gc(WW / CB, batch);
    const size_t smc = (size_t)(WW + CB * G::LP) * sizeof(float2);
    if (!inverse) {
      k_fft_rows<WW, false><<<gr, 256, smr, s>>>(d, nrows);
      k_fft_cols<WW, false><<<gc, 256, smc, s>>>(d, CB);
    } else {
      k_fft_rows<WW, true><<<gr, 256, smr, s>>>(d, nrows);
      k_fft_cols<WW, true><<<gc, 256, smc, s>>>(d, CB);
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_finite_check(const float* p, size_t n, int* flag, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_finite<<<296, 256, 0, s>>>(p, n, flag);
  return cudaGetLastError();
}


// ===================================================================== batch
// Many independent reconstructions in one persistent launch.  Each CTA takes
// the next task of a global list (atomic counter), waits until its problem
// has completed the tasks of all earlier passes (per-problem counter, acquire
// load), runs the pass body on its tiles, and counts the task done (release).
// The list interleaves the problems pass by pass, and every wait is for a
// task of a smaller index, so with all CTAs resident (cooperative launch) the
// schedule cannot deadlock; every wait is bounded anyway: past `timeout_ns`
// of the global timer the CTA records the problem in *error and all CTAs
// leave.
namespace {

PTY_D unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
PTY_D unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Not inlined: each pattern size keeps its own register allocation instead of
// one allocation for all of them inside the persistent kernel.
template <int W>
__device__ __noinline__ void batch_task(const BatchProb& pb, const BatchTask& tk) {
  const int* ids = pb.gpos + tk.ids_off;
  switch (tk.kind) {
    case BT_ROWS:
      for (int bx = tk.x0; bx < tk.x1; ++bx) {
        rows_fwd_body<W>(pb.O, pb.Hx, pb.P, pb.M, pb.R, pb.ppc, ids, pb.corners, tk.npatch,
                         pb.tw, pb.scratch, pb.omax_part, pb.M, 0, bx, tk.y);
        __syncthreads();
      }
      break;
    case BT_COLS:
      for (int bx = tk.x0; bx < tk.x1; ++bx) {
        cols_body<W, false>(pb.scratch, pb.M, pb.CB, pb.I, ids, pb.tw, pb.inv_w, pb.a.eps,
                            pb.err_part, pb.M, 0, 1, tk.npatch, bx, tk.y);
        __syncthreads();
      }
      break;
    case BT_ROWS_INV:
      for (int bx = tk.x0; bx < tk.x1; ++bx) {
        rows_inv_body<W>(pb.O, pb.Hx, pb.P, pb.M, pb.R, pb.ppc, ids, pb.corners, tk.npatch,
                         pb.scratch, pb.omax_part, pb.pmax_part, pb.n_pmax, pb.tw, pb.a, pb.pnum,
                         pb.pden, pb.osum, tk.flag, pb.M, 0, bx, tk.y);
        __syncthreads();
      }
      break;
    case BT_PROBE:
      for (int bx = tk.x0; bx < tk.x1; ++bx) {
        probe_apply_body(pb.P, pb.M, W * W, pb.pnum, pb.pden, pb.osum, tk.flag, pb.a.alpha_P,
                         pb.a.reg_eps, pb.pmax_part, bx, pb.n_pmax);
        __syncthreads();
      }
      break;
    default:
      err_reduce_body(pb.err_part, pb.err_part_n, pb.inv_sumI, pb.err_iter + tk.it);
      break;
  }
}

__global__ void __launch_bounds__(256)
k_batch(const BatchProb* __restrict__ probs, const BatchTask* __restrict__ tasks, int ntask,
        unsigned* next, unsigned* done, int* error, unsigned long long timeout_ns) {
  __shared__ int s_stop;
  __shared__ BatchProb s_pb;  // descriptor and task live in shared memory, not registers
  __shared__ BatchTask s_tk;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = (int)atomicAdd(next, 1u);
      int stop = 1;
      if (t < ntask) {
        stop = 0;
        const unsigned need = tasks[t].need;
        const unsigned* cnt = done + tasks[t].prob;
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(cnt) < need) {
          if (*(volatile int*)error) {
            stop = 1;
            break;
          }
          if (global_ns() - t0 > timeout_ns) {
            atomicCAS(error, 0, 1 + tasks[t].prob);
            stop = 1;
            break;
          }
          __nanosleep(128);
        }
        __threadfence();
      }
      s_stop = stop;
      if (!stop) {
        s_tk = tasks[t];
        s_pb = probs[s_tk.prob];
      }
    }
    __syncthreads();
    if (s_stop) break;
    switch (s_pb.W) {
      case 32: batch_task<32>(s_pb, s_tk); break;
      case 64: batch_task<64>(s_pb, s_tk); break;
      case 96: batch_task<96>(s_pb, s_tk); break;
      case 128: batch_task<128>(s_pb, s_tk); break;
      case 192: batch_task<192>(s_pb, s_tk); break;
      default: batch_task<256>(s_pb, s_tk); break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + s_tk.prob, 1u);
    }
    __syncthreads();  // s_tk / s_pb are rewritten by the next fetch
  }
}

}  // namespace

size_t batch_smem(const Tiling& t) { return std::max(std::max(t.smA, t.smB), t.smC); }

cudaError_t batch_grid(size_t smem, int* ctas) {
  cudaError_t e = allow_max_smem((const void*)k_batch);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, 256, smem)) != cudaSuccess)
    return e;
  *ctas = std::max(1, per) * sms;
  return cudaSuccess;
}

cudaError_t launch_batch(const BatchProb* probs, const BatchTask* tasks, int ntask,
                         unsigned* next, unsigned* done, int* error,
                         unsigned long long timeout_ns, int ctas, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch, probs, tasks, ntask, next, done, error, timeout_ns);
}

}  // namespace pty
