// Device bodies of the M-rPIE passes, shared by the per-pass kernels and the
// persistent batched kernel.  Equations are those of the M-rPIE section of
// Guzzi et al. (arXiv 2205.04295): exit waves (Eq. 1, per mode as in Eq. 4),
// far-field propagation (Eq. 2, unitary DFT), the mixed-state modulus
// constraint (Eq. 7), the object update (Eq. 6) and the probe update (Eq. 5).
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
#pragma once
#include "pty_copy.cuh"
#include "pty_fft.cuh"
#include "pty_internal.h"
#include "pty_pdl.cuh"

namespace pty {

namespace {


// Square root through the hardware reciprocal square root (rsqrtf, relative
// error about 2^-22, far below what the parity bars resolve); exact 0 at 0.
PTY_D float sqrt_rs(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

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
// Block-wide maximum; every thread gets the result.  Contains barriers.
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
// Request (cp.async) the crop rows [r0, r0 + R) of the patch with corner cc
// into `ost` (R x W, 16-byte aligned).  A crop row that starts on a 16-byte
// boundary moves in 16-byte pieces, any other (an odd corner column) in
// 8-byte pieces.
template <int W>
PTY_D void stage_crop_rows(const float2* O, int Hx, int2 cc, int R, int r0, float2* ost) {
  for (int r = 0; r < R; ++r) {
    const float2* src = O + (size_t)(cc.x + r0 + r) * Hx + cc.y;
    float2* dst = ost + r * W;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      for (int h = threadIdx.x; h < W / 2; h += blockDim.x) cp_async<16>(dst + 2 * h, src + 2 * h);
    } else {
      for (int c = threadIdx.x; c < W; c += blockDim.x) cp_async<8>(dst + c, src + c);
    }
  }
}
template <int W>
PTY_D void rows_fwd_stage(const float2* O, int Hx, int2 cc, int R, int r0, float2* ost) {
  stage_crop_rows<W>(O, Hx, cc, R, r0, ost);
}

// Barrier over a row line's L lanes: they are consecutive threads, so where
// lines tile warps (L = 8, 16) the warp suffices (every thread of the warp
// calls it); L = 12 lines straddle warps and take the CTA barrier.
template <int W>
PTY_D void line_sync() {
  if constexpr (32 % Line<W>::L == 0)
    __syncwarp();
  else
    __syncthreads();
}

// The next patch's crop rows are requested while the current patch is
// transformed (double-buffered in shared memory).  PSTAGE copies the CTA's
// probe rows to shared memory once; without it they are read at use through
// L1 (a few KB per CTA, cached), which leaves that shared memory free for more
// CTAs per SM.
template <int W, bool PSTAGE = true>
PTY_D void rows_fwd_body(const float2* O, int Hx, const float2* P,
           int M, int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           const float2* __restrict__ tw_g, float2* __restrict__ scratch,
           float* __restrict__ omax_part, int npl, int xo, int bx, int by) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* Prow = tw + W;                       // M x R x W probe rows (PSTAGE)
  float2* tbuf = Prow + (PSTAGE ? M * R * W : 0);
  float2* ost = tbuf + (M + xo) * R * G::LP;  // 2 x R x W crop rows
  int2* scor = reinterpret_cast<int2*>(ost + 2 * R * W);  // ppc corners

  const int r0 = bx * R;
  const int nrb = W / R;
  const int p0 = by * ppc, p1 = min(npatch, p0 + ppc);
  pdl_trigger();
  // the CTA's corners, once: no dependent index loads inside the patch loop
  for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) scor[t] = corners[ids[p0 + t]];
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  pdl_wait();  // O, P and the partial maxima belong to the previous kernels
  // this row block's crop-maximum partials start at 0 (non-negative floats
  // order as their bit patterns: the warps combine theirs by integer atomicMax)
  for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) omax_part[(size_t)(p0 + t) * nrb + bx] = 0.f;
  __syncthreads();
  if (p0 < p1) rows_fwd_stage<W>(O, Hx, scor[0], R, r0, ost);
  cp_async_commit();
  if constexpr (PSTAGE) {
    for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) {
      const int k = e / (R * W), rem = e - k * R * W, r = rem / W, c = rem - r * W;
      Prow[e] = P[((size_t)k * W + r0 + r) * W + c];
    }
  }

  // lines: (mode k, row r) for k < M, and with xo the crop itself as plane M
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < (M + xo) * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  for (int lp = p0; lp < p1; ++lp) {
    cp_async_wait<0>();
    __syncthreads();  // this patch's crop rows have landed; lbuf is free
    if (lp + 1 < p1)
      rows_fwd_stage<W>(O, Hx, scor[lp + 1 - p0], R, r0, ost + ((lp + 1 - p0) & 1) * R * W);
    cp_async_commit();
    float omax = 0.f;
    if (act && lane < G::N2) {
      const float2* prow = PSTAGE ? Prow + (k * R + r) * W
                                  : P + ((size_t)(k < M ? k : 0) * W + r0 + r) * W;
      const float2* orow = ost + ((lp - p0) & 1) * R * W + r * W;
      float2 v[G::N1];
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) {
        const int c = G::N2 * n1 + lane;
        const float2 o = orow[c];
        v[n1] = k < M ? cmul(PSTAGE ? prow[c] : __ldg(prow + c), o) : o;
        omax = fmaxf(omax, cabs2(o));
      }
      fwd_step1<W>(v, lane, tw, lbuf);
    }
    omax = warp_max(omax);
    if ((threadIdx.x & 31) == 0 && omax > 0.f)
      atomicMax(reinterpret_cast<int*>(omax_part + (size_t)lp * nrb + bx), __float_as_int(omax));
    line_sync<W>();  // the transpose stays within the line
    if (act && lane < G::N1) {
      float2 z[G::N2];
      fwd_step3<W>(z, lane, lbuf);
      float2* dst = scratch + (((size_t)lp * npl + k) * W + r0 + r) * W;
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = z[k2];
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- pass B
// Request (cp.async) the column block [c0, c0 + CB) of the MA planes of patch
// slot lp into `stage` ([plane][row][column]) and the block's counts into
// `cnt` ([row][column], rows and columns fftshifted, DC at the centre of the
// stored pattern).  CB is even, so every segment is 16-byte aligned.
// With a tensor map `tm` (planes of W x W complex over the scratch, box
// CB x W x 1), thread 0 requests the MA boxes by TMA, completing on `mbar`;
// without one, every thread issues 16-byte cp.async copies.
template <int W, int CB>
PTY_D void cols_stage(const float2* scratch, const uint16_t* I, int j, int lp, int npl, int MA,
                      int c0, float2* stage, uint16_t* cnt, const void* tm,
                      unsigned long long* mbar, int plane0 = 0) {
  if (tm) {
    if (threadIdx.x == 0) {
      fence_proxy_async();  // the stage was just read through the generic proxy
      mbar_expect_tx(mbar, (unsigned)(MA * W * CB * sizeof(float2)));
      for (int k = 0; k < MA; ++k)
        tma_load_3d(stage + k * W * CB, tm, c0, 0, plane0 + lp * npl + k, mbar);
    }
  } else {
    const int cpr = CB / 2;  // 16-byte chunks per row segment
    const int nch = MA * W * cpr;
    for (int i = threadIdx.x; i < nch; i += blockDim.x) {
      const int h = i % cpr, row = i / cpr;  // row = plane * W + u
      const int k = row / W, u = row - k * W;
      cp_async<16>(stage + row * CB + 2 * h,
                   scratch + (((size_t)lp * npl + k) * W + u) * W + c0 + 2 * h);
    }
  }
  // CB consecutive counts per detector row; CB divides W/2, so the block of
  // shifted columns does not wrap
  const uint16_t* Ij = I + (size_t)j * W * W + (c0 + W / 2) % W;
  if constexpr (CB >= 8) {
    constexpr int q = CB / 8;  // 16-byte chunks per row
    for (int i = threadIdx.x; i < W * q; i += blockDim.x) {
      const int u = i / q, h = i - u * q;
      cp_async<16>(cnt + u * CB + 8 * h, Ij + (size_t)((u + W / 2) % W) * W + 8 * h);
    }
  } else if constexpr (CB == 4) {
    for (int u = threadIdx.x; u < W; u += blockDim.x)
      cp_async<8>(cnt + u * 4, Ij + (size_t)((u + W / 2) % W) * W);
  } else {
    for (int u = threadIdx.x; u < W; u += blockDim.x)
      cp_async<4>(cnt + u * 2, Ij + (size_t)((u + W / 2) % W) * W);
  }
}

// Barrier over the threads of one mode's CB column lines (CB * L consecutive
// threads: the transposes of a line never leave its mode).  Warp-aligned
// groups of two or more warps take named barrier 1 + k; a warp, or groups
// that tile a warp, __syncwarp (every thread of the warp calls it); anything
// else the whole CTA.  With CB * L a multiple of 32 the launch has exactly
// M * CB * L threads, so every participant of barrier 1 + k is in mode k.
template <int W, int CB>
PTY_D void mode_sync(int k) {
  constexpr int n = CB * Line<W>::L;
  if constexpr (n % 32 == 0 && n > 32)
    asm volatile("bar.sync %0, %1;" ::"r"(1 + k), "r"(n) : "memory");
  else if constexpr (n == 32 || (n < 32 && 32 % n == 0))
    __syncwarp();
  else
    __syncthreads();
}

// GRAD = false: the modulus constraint (Eq. 7); with xb >= 0 (XCORR_B
// registration) also the model intensity S = sum_p |Psi_p|^2 and the counts,
// written unshifted into the real parts of scratch planes xb and xb + 1.  GRAD = true: the Fourier-
// domain step of the amplitude-loss adjoint, G_Psi = 2 (1 - sqrt(I) / A) Psi
// with A = sqrt(S + eps) (eps carries delta), and the loss partial sums.
// The next patch's column block is requested while the current one is
// transformed (double-buffered counts, one stage for the far field: it is
// refilled once its values are in registers).  STAGE = false (the batched
// form, one patch per call, where a prefetch has nothing to overlap) reads
// the columns straight into registers and needs no stage.  CB is a
// compile-time constant: with a run-time CB the per-element shared-memory
// offsets are hoisted out of the patch loop and spill.
template <int W, int CB, bool GRAD, bool STAGE = true>
PTY_D void cols_body(float2* __restrict__ scratch, int M,
       const uint16_t* __restrict__ I, const int* __restrict__ ids,
       const float2* __restrict__ tw_g, float inv_w, float eps,
       float* __restrict__ err_part, int npl, int ppcb, int npatch, int bx, int by,
       const void* tm = nullptr, int* err = nullptr, int xb = -1, int plane0 = 0) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  __shared__ __align__(8) unsigned long long mbar;
  float2* tw = reinterpret_cast<float2*>(smem4);
  // M x W x CB, 128-byte aligned (TMA destination; every plane's slice
  // W * CB * 8 bytes is a multiple of 128)
  float2* stage = reinterpret_cast<float2*>(
      (reinterpret_cast<uintptr_t>(tw + W) + 127) & ~static_cast<uintptr_t>(127));
  float2* tbuf = stage + (STAGE ? M * W * CB : 0);               // M x CB lines
  float* Sb = reinterpret_cast<float*>(tbuf + M * CB * G::LP);   // M x W x CB
  uint16_t* cnt = reinterpret_cast<uint16_t*>(Sb + M * CB * W);  // 2 x W x CB
  int* sids = reinterpret_cast<int*>(cnt + 2 * W * CB);           // ppcb pattern ids
  __shared__ float red[32];

  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  const int c0 = bx * CB;
  const int c = threadIdx.x % CB, rest = threadIdx.x / CB;
  const int lane = rest % G::L, k = rest / G::L;
  const bool act = k < M;  // thread of mode k's line for column c
  const int kk0 = act ? k : 0;
  float2* lbuf = tbuf + (kk0 * CB + c) * G::LP;
  const float2* srow = stage + kk0 * W * CB + c;
  const int nw = (blockDim.x + 31) >> 5;
  const int p0 = by * ppcb, p1 = min(npatch, p0 + ppcb);
  const bool tma = STAGE && tm != nullptr;
  unsigned phase = 0;
  pdl_trigger();
  for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) sids[t] = ids[p0 + t];
  if (tma && threadIdx.x == 0) mbar_init(&mbar, 1 + stalled_arrivals(err));
  pdl_wait();  // the far field comes from pass A
  __syncthreads();
  if constexpr (STAGE) {
    if (p0 < p1)
      cols_stage<W, CB>(scratch, I, sids[0], p0, npl, M, c0, stage, cnt, tm, &mbar, plane0);
    cp_async_commit();
  }
  for (int lp = p0; lp < p1; ++lp) {
    const int j = sids[lp - p0];
    const uint16_t* cn = cnt + (STAGE ? ((lp - p0) & 1) * W * CB : 0);
    float2* col = scratch + ((size_t)lp * npl + kk0) * W * W + c0 + c;
    if constexpr (STAGE) {
      bool ok = true;
      if (tma) {
        // every thread waits on the mbarrier itself, so the TMA-written block
        // is visible to it; its own count copies land with cp_async_wait (the
        // others' are read after a later CTA barrier); the lines' buffers are
        // free once the mode's threads have left the previous inverse step B
        ok = mbar_wait_bounded(&mbar, phase, 200000000ull);  // 0.2 s of the global timer
        phase ^= 1;
        cp_async_wait<0>();
        mode_sync<W, CB>(k);
      } else {
        cp_async_wait<0>();
        __syncthreads();  // this patch's block has landed
      }
      if (act && lane < G::N2) {
        float2 v[G::N1];
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = srow[(G::N2 * n1 + lane) * CB];
        fwd_step1<W>(v, lane, tw, lbuf);
      }
      // the stage is free: request the next patch.  With TMA a wait that ran
      // out makes every thread leave here (uniformly: none waits at a barrier
      // afterwards); what it read from the stage is discarded.
      if (tma) {
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0 && err) atomicExch(err, 1);
          if (!ok) mbar_wait_bounded(&mbar, phase ^ 1, 200000000ull);  // the copy in flight
          return;
        }
      } else {
        __syncthreads();
      }
      if (lp + 1 < p1)
        cols_stage<W, CB>(scratch, I, sids[lp + 1 - p0], lp + 1, npl, M, c0, stage,
                          cnt + ((lp + 1 - p0) & 1) * W * CB, tm, &mbar, plane0);
      cp_async_commit();
    } else {
      // the counts and the columns are requested together: one round trip
      float2 v[G::N1];
      if (act && lane < G::N2) {
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = col[(size_t)(G::N2 * n1 + lane) * W];
      }
      {
        const uint16_t* Ij = I + (size_t)j * W * W + (c0 + W / 2) % W;
        for (int el = threadIdx.x; el < CB * W; el += blockDim.x) {
          const int u = el / CB, cl = el - u * CB;
          cnt[el] = __ldcs(Ij + (size_t)((u + W / 2) % W) * W + cl);
        }
      }
      __syncthreads();  // tw (first patch); the previous patch's reads of lbuf
      if (act && lane < G::N2) fwd_step1<W>(v, lane, tw, lbuf);
      __syncthreads();
    }
    float2 z[G::N2];
    if (act && lane < G::N1) {
      fwd_step3<W>(z, lane, lbuf);
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2) Sb[(k * W + lane + G::N1 * k2) * CB + c] = cabs2(z[k2]);
    }
    __syncthreads();
    // constraint factor once per detector pixel (u, c): S = sum_k |Psi_k|^2 in a
    // fixed mode order, f = sqrt(I) / (sqrt(S) + eps) folded with both 1/W
    // normalisations; stored over mode 0's |Psi|^2.
    float e = 0.f;
    {
      const float f2 = inv_w * inv_w;
      // two detector pixels per step: their mode sums are loaded before
      // either factor is stored (the store may alias the next loads)
      const int n = CB * W, st = blockDim.x;
      for (int el0 = threadIdx.x; el0 < n; el0 += 2 * st) {
        const bool two = el0 + st < n;
        float s2[2] = {0.f, 0.f};
        float c2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int el = el0 + h * st;
          if (h == 0 || two) {
            const int u = el / CB, cl = el - u * CB;
#pragma unroll 4
            for (int kk = 0; kk < M; ++kk) s2[h] += Sb[(kk * W + u) * CB + cl];
            c2[h] = (float)cn[el];
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !two) break;
          const int el = el0 + h * st;
          const int u = el / CB, cl = el - u * CB;
          const float s = s2[h];
          const float sI = sqrt_rs(c2[h]);
          if (!GRAD) {
            // rounded products and sums written out (no contraction), as in
            // the fused patch kernel
            const float a = __fmul_rn(sqrt_rs(s), inv_w);
            const float d = __fsub_rn(a, sI);
            e = fmaf(d, d, e);
            // quotient by a reciprocal-multiply (within 2 ulp of the division)
            Sb[u * CB + cl] = __fmul_rn(__fdividef(sI, __fadd_rn(a, eps)), f2);
            if (xb >= 0) {
              // XCORR_B: the model intensity and the counts, unshifted, as the
              // real parts of scratch planes xb and xb + 1
              float2* pl = scratch + ((size_t)lp * npl + xb) * W * W + (size_t)u * W + c0 + cl;
              pl[0] = make_float2(s * f2, 0.f);
              pl[(size_t)W * W] = make_float2(c2[h], 0.f);
            }
          } else {
            const float a = sqrt_rs(fmaf(s, f2, eps));
            const float d = a - sI;
            e = fmaf(d, d, e);
            Sb[u * CB + cl] = 2.f * (1.f - __fdividef(sI, a)) * f2;
          }
        }
      }
    }
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x >= blockDim.x - 32) {
      // the last warp sums the warp partials (a fixed shuffle tree)
      const int l = threadIdx.x & 31;
      const float t = warp_sum(l < nw ? red[l] : 0.f);
      if (l == 0) err_part[(size_t)j * (W / CB) + bx] = t;
    }
    if (act && lane < G::N1) {
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2)
        z[k2] = cscale(z[k2], Sb[(lane + G::N1 * k2) * CB + c]);
      inv_stepA<W>(z, lane, tw, lbuf);
    }
    // the transpose stays within the mode's lines; the batched form (one
    // patch per call, inside a persistent kernel) keeps the CTA barrier
    if constexpr (STAGE)
      mode_sync<W, CB>(k);
    else
      __syncthreads();
    if (act && lane < G::N2) {
      float2 v[G::N1];
      inv_stepB<W>(v, lane, lbuf);
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) col[(size_t)(G::N2 * n1 + lane) * W] = v[n1];
    }
  }
  if constexpr (STAGE) cp_async_wait<0>();
}


// ---------------------------------------------------------------- pass C
// Request patch slot lp's far-field rows [r0, r0 + R) of the M modes into
// `zst` ([mode][row][column]) (rows_inv_stage_far), and with rows_inv_stage
// also its crop rows into `ost`.  With `mbar`, thread 0 moves the far-field
// rows by bulk copies (one per row, completing on the mbarrier); otherwise
// every thread issues 16-byte cp.async copies.  The crop rows (any
// alignment) always take cp.async.
template <int W>
PTY_D void rows_inv_stage_far(const float2* scratch, int lp, int npl, int M, int R, int r0,
                              float2* zst, unsigned long long* mbar) {
  if (mbar) {
    if (threadIdx.x == 0) {
      fence_proxy_async();  // the stage was just read through the generic proxy
      mbar_expect_tx(mbar, (unsigned)(M * R * W * sizeof(float2)));
      for (int line = 0; line < M * R; ++line) {  // line = mode * R + row
        const int k = line / R, r = line - k * R;
        bulk_load(zst + line * W, scratch + (((size_t)lp * npl + k) * W + r0 + r) * W,
                  (unsigned)(W * sizeof(float2)), mbar);
      }
    }
  } else {
    constexpr int hw = W / 2;  // 16-byte chunks per row
    for (int i = threadIdx.x; i < M * R * hw; i += blockDim.x) {
      const int line = i / hw, h = i - line * hw;  // line = mode * R + row
      const int k = line / R, r = line - k * R;
      cp_async<16>(zst + line * W + 2 * h,
                   scratch + (((size_t)lp * npl + k) * W + r0 + r) * W + 2 * h);
    }
  }
}
template <int W>
PTY_D void rows_inv_stage(const float2* scratch, const float2* O, int Hx, int2 cc, int lp,
                          int npl, int M, int R, int r0, float2* zst, float2* ost,
                          unsigned long long* mbar) {
  rows_inv_stage_far<W>(scratch, lp, npl, M, R, r0, zst, mbar);
  stage_crop_rows<W>(O, Hx, cc, R, r0, ost);
}

// A lane's object-update terms for its N1 pixels of one (mode, row) line:
// D = psi' - P o, T = D conj(P) into the CTA's term buffer, nm += D conj(o).
// PMODE: the probe values from registers (0), a shared-memory row (1) or a
// global row through L1 (2).  The pointers do not alias, which lets every
// load be issued ahead of the term stores.
template <int W, int PMODE>
PTY_D void upd_terms(const float2* v, const float2* pk, const float2* __restrict__ orow,
                     const float2* __restrict__ prow, float2* __restrict__ T, float2* nm,
                     int lane) {
  using G = Line<W>;
#pragma unroll
  for (int n1 = 0; n1 < G::N1; ++n1) {
    const int c = G::N2 * n1 + lane;
    const float2 o = orow[c];
    const float2 pkv = PMODE == 0 ? pk[n1] : PMODE == 1 ? prow[c] : __ldg(prow + c);
    const float2 D = csub(v[n1], cmul(pkv, o));
    T[c] = cmulc(D, pkv);
    nm[n1] = cadd(nm[n1], cmulc(D, o));
  }
}

// The object update of the CTA's R rows (Eq. 6, sum of the modes' terms in
// mode order) and the denominator sums, two pixels per step with their loads
// issued before either pixel's stores.
PTY_D void upd_object(int R, int W, int M, const float2* __restrict__ oc,
                      const float2* __restrict__ tb, const float* __restrict__ invd,
                      float* __restrict__ den, float2* __restrict__ O, int Hx, int2 cc, int r0,
                      float2* __restrict__ onew, bool refine, float omb, float bom) {
  const int n = R * W, st = blockDim.x;
  for (int e0 = threadIdx.x; e0 < n; e0 += 2 * st) {
    const bool two = e0 + st < n;
    float2 o2[2], s2[2];
    float sc2[2], d2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 0 || two) {
        const int e = e0 + h * st, rr = e / W, c = e - rr * W;
        o2[h] = oc[e];
        float2 sm = make_float2(0.f, 0.f);
        for (int kk = 0; kk < M; ++kk) sm = cadd(sm, tb[(kk * R + rr) * W + c]);
        s2[h] = sm;
        sc2[h] = invd[e];
        d2[h] = den[e];
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
      const int e = e0 + h * st, rr = e / W, c = e - rr * W;
      const float2 o = o2[h];
      const float2 onw = make_float2(fmaf(sc2[h], s2[h].x, o.x), fmaf(sc2[h], s2[h].y, o.y));
      O[(size_t)(cc.x + r0 + rr) * Hx + cc.y + c] = onw;
      if (refine) onew[e] = onw;
      den[e] = d2[h] + fmaf(omb, cabs2(o), bom);
    }
  }
}

// The next patch's far-field and crop rows are requested while the current
// patch is transformed: no registers wait on global loads.  A lane always
// owns the same W / N2 pixels of its (mode, row) line, so its probe-numerator
// sums stay in registers across the patches; its probe values are read at use,
// which keeps the kernel within 128 registers without spilling (holding them
// in registers cost 5 % of this pass).  With PSTAGE they come from the CTA's
// probe rows, copied to shared memory once in the prologue (the probe is
// constant during the pass; 5 % faster than reading them through L1 at use),
// which the tiling turns on only where the extra shared memory costs no CTA
// per SM (at 256², 4 modes it would cost one: 15 % slower).  PK_REG holds
// them in registers anyway: the batched form's task function, compiled on
// its own, measured 1-2.5 % faster that way.
template <int W, bool PK_REG = false, bool PSTAGE = false>
PTY_D void rows_inv_body(float2* O, int Hx, const float2* P, int M,
           int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           float2* scratch, const float* omax_part,
           const float* pmax_part, int n_pmax,
           const float2* __restrict__ tw_g, UpdArgs a,
           float2* pnum, float* pden,
           float* osum, int accumulate, int npl, int refine, int bx, int by,
           int* err = nullptr) {
  using G = Line<W>;
  extern __shared__ float4 smem4[];
  __shared__ __align__(8) unsigned long long mbar_s;
  unsigned long long* mbar = err ? &mbar_s : nullptr;  // bulk copies with error reporting
  unsigned phase = 0;
  const int TB = max(M * R * G::LP, M * R * W);
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;             // transpose buffer, then D conj(P) terms
  float2* ostash = tbuf + TB;        // 2 x R x W: crop rows, double-buffered
  float2* zst = ostash + 2 * R * W;  // M x R x W far-field rows
  float2* prs = zst + M * R * W;     // M x R x W probe rows (PSTAGE only)
  float* invd = reinterpret_cast<float*>(prs + (PSTAGE ? M * R * W : 0));  // alpha_O / den.
  float* den = invd + R * W;
  int2* scor = reinterpret_cast<int2*>(den + R * W);         // ppc corners
  float* som = reinterpret_cast<float*>(scor + ppc);         // ppc crop maxima
  __shared__ float s_pmax;

  const int r0 = bx * R;
  const int nrb = W / R;
  pdl_trigger();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  if (mbar && threadIdx.x == 0) mbar_init(mbar, 1 + stalled_arrivals(err));
  pdl_wait();  // everything below is written by earlier kernels
  const int p0 = by * ppc, p1 = min(npatch, p0 + ppc);
  // the first patch's far-field rows need no corner: they are requested
  // before the prologue's loads, its crop rows once the corners are in
  if (p0 < p1) rows_inv_stage_far<W>(scratch, p0, npl, M, R, r0, zst, mbar);
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int i = threadIdx.x; i < n_pmax; i += 32) m = fmaxf(m, pmax_part[i]);
    m = warp_max(m);
    if (threadIdx.x == 0) s_pmax = m;
  }
  __syncthreads();
  {
    const float pmax = s_pmax;
    const float gden = fmaf(a.gamma, pmax, a.reg_eps * pmax);  // one rounding, as in every kernel
    for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
      const int rr = e / W, c = e - rr * W;
      float s = 0.f;
      for (int k = 0; k < M; ++k) {
        const float2 p = P[((size_t)k * W + r0 + rr) * W + c];
        if constexpr (PSTAGE) prs[(k * R + rr) * W + c] = p;
        s += cabs2(p);
      }
      const float dn = fmaf(1.f - a.gamma, s, gden);
      invd[e] = dn > 0.f ? a.alpha_O / dn : 0.f;  // a zero denominator has a zero numerator
      den[e] = 0.f;
    }
  }

  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < M * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  const bool own = act && lane < G::N2;  // holds pixels c = N2 n1 + lane
  float2 nm[G::N1], pk[G::N1];
  const float2* prow = P + ((size_t)k * W + r0 + r) * W;
#pragma unroll
  for (int n1 = 0; n1 < G::N1; ++n1) {
    nm[n1] = make_float2(0.f, 0.f);
    if constexpr (PK_REG) pk[n1] = own ? prow[G::N2 * n1 + lane] : make_float2(0.f, 0.f);
  }
  // the CTA's corners and crop maxima max_r |o_j|^2 (reduced over the row
  // blocks of pass A), once: no dependent global loads inside the patch loop
  {
    const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) scor[t] = corners[ids[p0 + t]];
    for (int t = w; t < p1 - p0; t += nw) {
      float m = 0.f;
      for (int i = l; i < nrb; i += 32) m = fmaxf(m, omax_part[(size_t)(p0 + t) * nrb + i]);
      m = warp_max(m);
      if (l == 0) som[t] = m;
    }
  }
  __syncthreads();
  float osum_local = 0.f;
  if (p0 < p1) stage_crop_rows<W>(O, Hx, scor[0], R, r0, ostash);
  cp_async_commit();
  for (int lp = p0; lp < p1; ++lp) {
    const int2 cc = scor[lp - p0];
    const float2* oc = ostash + ((lp - p0) & 1) * R * W;
    bool ok = true;
    if (mbar) {
      ok = mbar_wait_bounded(mbar, phase, 200000000ull);  // 0.2 s of the global timer
      phase ^= 1;
    }
    cp_async_wait<0>();
    if (__syncthreads_or(!ok)) {  // this patch's rows have landed, or the CTA leaves
      if (threadIdx.x == 0) atomicExch(err, 1);
      if (!ok) mbar_wait_bounded(mbar, phase ^ 1, 200000000ull);  // the copy in flight
      return;
    }
    if (act && lane < G::N1) {
      float2 z[G::N2];
      const float2* src = zst + (k * R + r) * W;
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = src[lane + G::N1 * k2];
      inv_stepA<W>(z, lane, tw, lbuf);
    }
    __syncthreads();  // the far-field stage is free: request the next patch
    if (lp + 1 < p1)
      rows_inv_stage<W>(scratch, O, Hx, scor[lp + 1 - p0], lp + 1, npl, M, R, r0, zst,
                        ostash + ((lp + 1 - p0) & 1) * R * W, mbar);
    cp_async_commit();
    float2 v[G::N1];
    if (act && lane < G::N2) inv_stepB<W>(v, lane, lbuf);
    __syncthreads();  // tbuf is reused below for the D conj(P) terms
    if (own) {
      float2* T = tbuf + (k * R + r) * W;
      constexpr int PMODE = PK_REG ? 0 : PSTAGE ? 1 : 2;
      upd_terms<W, PMODE>(v, pk, oc + r * W, PSTAGE ? prs + (k * R + r) * W : prow, T, nm, lane);
    }
    __syncthreads();
    const float om = som[lp - p0];
    // with XCORR_A the refined crop rows o'_j go, untransformed, to plane
    // M + 1 (the registration takes their row DFTs for a batch of groups)
    upd_object(R, W, M, oc, tbuf, invd, den, O, Hx, cc, r0,
               refine ? scratch + (((size_t)lp * npl + M + 1) * W + r0) * W : nullptr, refine,
               1.f - a.beta, a.beta * om);
    osum_local += om;
    // the next patch's first barrier orders these reads of tbuf before its
    // transpose writes
  }
  cp_async_wait<0>();
  const int slot = by;
  if (own) {
    float2* dst = pnum + (((size_t)slot * M + k) * W + r0 + r) * W;
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) {
      const int c = G::N2 * n1 + lane;
      dst[c] = accumulate ? cadd(dst[c], nm[n1]) : nm[n1];
    }
  }
  for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
    const int rr = e / W, c = e - rr * W;
    const size_t g = ((size_t)slot * W + r0 + rr) * W + c;
    pden[g] = accumulate ? pden[g] + den[e] : den[e];
  }
  if (bx == 0 && threadIdx.x == 0)
    osum[slot] = accumulate ? osum[slot] + osum_local : osum_local;
}

// ------------------------------------------------------------- probe apply
PTY_D void probe_apply_body(float2* P, int M, int WW, const float2* pnum, const float* pden,
                            const float* osum, int nslots, float alpha_P, float reg_eps,
                            float* pmax_part, int bx, int gx) {
  __shared__ float red[32];
  pdl_trigger();
  pdl_wait();
  float os = 0.f;
  for (int s = 0; s < nslots; ++s) os += osum[s];
  const float guard = reg_eps * os;
  float lmax = 0.f;
  // The slot sums run in slot order; their loads are issued eight slots at a
  // time (independent loads in flight instead of one L2 round trip per slot).
  constexpr int kB = 8;
  for (int pix = bx * blockDim.x + threadIdx.x; pix < WW; pix += gx * blockDim.x) {
    float d = 0.f;
    for (int s0 = 0; s0 < nslots; s0 += kB) {
      float dv[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u)
        dv[u] = s0 + u < nslots ? pden[(size_t)(s0 + u) * WW + pix] : 0.f;
#pragma unroll
      for (int u = 0; u < kB; ++u)
        if (s0 + u < nslots) d += dv[u];
    }
    const float dd = d + guard;
    const float sc = dd > 0.f ? alpha_P / dd : 0.f;  // zero numerator too
    float pint = 0.f;
    for (int k = 0; k < M; ++k) {
      float2 n = make_float2(0.f, 0.f);
      for (int s0 = 0; s0 < nslots; s0 += kB) {
        float2 nv[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u)
          nv[u] = s0 + u < nslots ? pnum[((size_t)(s0 + u) * M + k) * WW + pix]
                                  : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kB; ++u)
          if (s0 + u < nslots) n = cadd(n, nv[u]);
      }
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

// Needs blockDim.x doubles of dynamic shared memory (a static array would be
// reserved in the persistent kernel for every task).
// The normalisation is 1 / sum(I): inv_sumI, or, when sum_dev is given, the
// device-resident counts sum (so that no host value waits for an upload).
template <typename T>
PTY_D void err_reduce_body(const T* part, size_t n, double inv_sumI,
                           const unsigned long long* sum_dev, float* out) {
  extern __shared__ float4 smem4[];
  double* red = reinterpret_cast<double*>(smem4);
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double inv = inv_sumI;
    if (sum_dev) inv = *sum_dev ? 1.0 / (double)*sum_dev : 0.0;
    *out = (float)(red[0] * inv);
  }
}

}  // namespace

}  // namespace pty
