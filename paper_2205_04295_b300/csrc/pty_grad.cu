// Differentiable forward model and its hand-written adjoint.
//
// Forward model (bilinear crop so that positions are differentiable; Eqs. 1,
// 2 and 4 of Guzzi et al., arXiv 2205.04295, with the amplitude loss):
//   o_j(r)  = sum_{a,b} w_a(fy) w_b(fx) O(iy + r_y + a, ix + r_x + b)
//   Psi_jp  = F(P_p o_j),  A_j = sqrt(sum_p |Psi_jp|^2 + delta)
//   L       = sum_j sum_u (A_j - sqrt(I_j))^2
// Adjoint, in PyTorch's convention for complex tensors (dL/dRe + i dL/dIm):
//   G_Psi = 2 (1 - sqrt(I)/A) Psi,  G_psi = F^-1 G_Psi,
//   dL/dP_p += conj(o_j) G_psi_p,   G_o = sum_p conj(P_p) G_psi_p,
//   dL/dO   += bilinear transpose of G_o,
//   dL/dy_j  = Re sum_r conj(G_o) do_j/dy (likewise x).
// The far field is recomputed per patch (no exit waves are stored):
//   grad_rows_fwd -> cols<GRAD> -> grad_rows_inv -> grad_scatter
// per chunk of a group of positions whose (W+1)-boxes are pairwise disjoint,
// so the scatter of dL/dO needs no atomics and is deterministic.
#include "pty_copy.cuh"
#include "pty_fft.cuh"
#include "pty_internal.h"
#include "pty_pdl.cuh"

#include <algorithm>

namespace pty {

namespace {

PTY_D float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Barrier over a row line's L lanes: consecutive threads, so where lines tile
// warps (L = 8, 16) the warp suffices (every thread of the warp calls it);
// L = 12 lines straddle warps and take the CTA barrier.
template <int W>
PTY_D void grad_line_sync() {
  if constexpr (32 % Line<W>::L == 0)
    __syncwarp();
  else
    __syncthreads();
}

struct Bil {
  int iy, ix;
  float fy, fx;
};
PTY_D Bil bil_of(const float* pos, int j) {
  Bil b;
  const float y = pos[2 * j], x = pos[2 * j + 1];
  b.iy = (int)floorf(y);
  b.ix = (int)floorf(x);
  b.fy = y - (float)b.iy;
  b.fx = x - (float)b.ix;
  return b;
}

// Request (cp.async) the R + 1 object rows iy + r0 .. iy + r0 + R, columns
// ix .. ix + W, that the bilinear crop rows r0 .. r0 + R - 1 of a patch read.
template <int W>
PTY_D void grad_stage(const float2* O, int Hx, const Bil& b, int R, int r0, float2* st) {
  constexpr int SP = W + 1;
  for (int e = threadIdx.x; e < (R + 1) * SP; e += blockDim.x) {
    const int q = e / SP, c = e - q * SP;
    cp_async<8>(st + e, O + (size_t)(b.iy + r0 + q) * Hx + b.ix + c);
  }
}

// o(r, c) and its derivatives from the staged rows (pitch W + 1).
template <int W>
PTY_D void bil_staged(const float2* st, const Bil& b, int r, int c, float2& o,
                      float2* dy = nullptr, float2* dx = nullptr) {
  constexpr int SP = W + 1;
  const float2* p = st + r * SP + c;
  const float2 q00 = p[0], q01 = p[1], q10 = p[SP], q11 = p[SP + 1];
  const float wy0 = 1.f - b.fy, wy1 = b.fy, wx0 = 1.f - b.fx, wx1 = b.fx;
  o.x = wy0 * (wx0 * q00.x + wx1 * q01.x) + wy1 * (wx0 * q10.x + wx1 * q11.x);
  o.y = wy0 * (wx0 * q00.y + wx1 * q01.y) + wy1 * (wx0 * q10.y + wx1 * q11.y);
  if (dy) {
    dy->x = wx0 * (q10.x - q00.x) + wx1 * (q11.x - q01.x);
    dy->y = wx0 * (q10.y - q00.y) + wx1 * (q11.y - q01.y);
    dx->x = wy0 * (q01.x - q00.x) + wy1 * (q11.x - q10.x);
    dx->y = wy0 * (q01.y - q00.y) + wy1 * (q11.y - q10.y);
  }
}

// ---------------------------------------------------- forward rows
// The next patch's object rows are requested while the current patch is
// transformed; the crop rows are interpolated once per patch (not once per
// mode).
template <int W>
__global__ void __launch_bounds__(256)
k_grad_rows_fwd(const float2* __restrict__ O, int Hx, const float2* __restrict__ P, int M,
                int R, int ppc, const int* __restrict__ ids, const float* __restrict__ pos,
                int npatch, const float2* __restrict__ tw_g, float2* __restrict__ scratch,
                int npl) {
  using G = Line<W>;
  constexpr int SP = W + 1;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* Prow = tw + W;
  float2* tbuf = Prow + M * R * W;
  float2* obuf = tbuf + M * R * G::LP;  // R x W interpolated crop rows
  float2* st = obuf + R * W;            // 2 x (R + 1) x (W + 1) object rows
  Bil* sb = reinterpret_cast<Bil*>(st + 2 * (R + 1) * SP);  // ppc crop geometries
  const int r0 = blockIdx.x * R;
  const int p0 = blockIdx.y * ppc, p1 = min(npatch, p0 + ppc);
  pdl_trigger();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  pdl_wait();  // positions, object and probe may come from the previous kernel
  // the CTA's crop geometries, once: no dependent loads inside the patch loop
  for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) sb[t] = bil_of(pos, ids[p0 + t]);
  __syncthreads();
  if (p0 < p1) grad_stage<W>(O, Hx, sb[0], R, r0, st);
  cp_async_commit();
  for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) {
    const int k = e / (R * W), rem = e - k * R * W, r = rem / W, c = rem - r * W;
    Prow[e] = P[((size_t)k * W + r0 + r) * W + c];
  }
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < M * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  for (int lp = p0; lp < p1; ++lp) {
    const Bil b = sb[lp - p0];
    const float2* sc = st + ((lp - p0) & 1) * (R + 1) * SP;
    cp_async_wait<0>();
    __syncthreads();  // this patch's rows have landed; obuf and lbuf are free
    if (lp + 1 < p1)
      grad_stage<W>(O, Hx, sb[lp + 1 - p0], R, r0, st + ((lp + 1 - p0) & 1) * (R + 1) * SP);
    cp_async_commit();
    for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
      const int rr = e / W, c = e - rr * W;
      bil_staged<W>(sc, b, rr, c, obuf[e]);
    }
    __syncthreads();
    if (act && lane < G::N2) {
      float2 v[G::N1];
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) {
        const int c = G::N2 * n1 + lane;
        v[n1] = cmul(Prow[(k * R + r) * W + c], obuf[r * W + c]);
      }
      fwd_step1<W>(v, lane, tw, lbuf);
    }
    grad_line_sync<W>();  // the transpose stays within the line
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

// ---------------------------------------------------- inverse rows + adjoint
// The far-field rows and the object rows of the next patch are requested
// (cp.async) while the current patch is transformed, so no register waits on
// a global load; the probe values are read at use through L1 (the CTA's
// rows of P, a few KB, stay cached), which leaves their shared memory to the
// far-field stage.
template <int W>
__global__ void __launch_bounds__(256)
k_grad_rows_inv(const float2* __restrict__ O, int Hx, const float2* __restrict__ P, int M,
                int R, int ppc, const int* __restrict__ ids, const float* __restrict__ pos,
                int npatch, float2* __restrict__ scratch, int npl,
                const float2* __restrict__ tw_g, float2* __restrict__ gP_part, int accumulate,
                float* __restrict__ gpos_part) {
  using G = Line<W>;
  constexpr int SP = W + 1;
  extern __shared__ float4 smem4[];
  const int TB = max(M * R * G::LP, M * R * W);
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* zst = tw + W;             // M x R x W far-field rows of the patch
  float2* tbuf = zst + M * R * W;   // transpose buffer, then conj(P) G_psi terms
  float2* gp = tbuf + TB;           // dL/dP partial sums of this CTA
  float2* obuf = gp + M * R * W;    // R x W interpolated crop rows
  float2* st = obuf + R * W;        // 2 x (R + 1) x (W + 1) object rows
  Bil* sb = reinterpret_cast<Bil*>(st + 2 * (R + 1) * SP);  // ppc crop geometries
  int* sj = reinterpret_cast<int*>(sb + ppc);                // ppc pattern ids
  // per patch and warp, the warp's (dL/dy, dL/dx) share: summed over the
  // warps in a fixed order once after the patch loop, so the patches need no
  // block reduction of their own
  float* gw = reinterpret_cast<float*>(sj + ppc);            // ppc x 8 x 2
  const int r0 = blockIdx.x * R, nrb = W / R;
  const int p0 = blockIdx.y * ppc, p1 = min(npatch, p0 + ppc);
  pdl_trigger();
  pdl_wait();  // the far field comes from the column pass
  for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) {
    sj[t] = ids[p0 + t];
    sb[t] = bil_of(pos, sj[t]);
  }
  __syncthreads();
  // patch q's object rows into stq and its far-field rows (16-byte pieces) into zst
  auto stage = [&](int q, float2* stq) {
    grad_stage<W>(O, Hx, sb[q - p0], R, r0, stq);
    constexpr int hw = W / 2;
    for (int i = threadIdx.x; i < M * R * hw; i += blockDim.x) {
      const int line = i / hw, h = i - line * hw;  // line = mode * R + row
      const int kk = line / R, rr = line - kk * R;
      cp_async<16>(zst + line * W + 2 * h,
                   scratch + (((size_t)q * npl + kk) * W + r0 + rr) * W + 2 * h);
    }
  };
  if (p0 < p1) stage(p0, st);
  cp_async_commit();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = tw_g[e];
  for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) gp[e] = make_float2(0.f, 0.f);
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < M * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  for (int lp = p0; lp < p1; ++lp) {
    const Bil b = sb[lp - p0];
    const float2* sc = st + ((lp - p0) & 1) * (R + 1) * SP;
    cp_async_wait<0>();
    __syncthreads();  // this patch's object and far-field rows have landed
    if (act && lane < G::N1) {
      const float2* src = zst + (k * R + r) * W;
      float2 z[G::N2];
#pragma unroll
      for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = src[lane + G::N1 * k2];
      inv_stepA<W>(z, lane, tw, lbuf);
    }
    for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
      const int rr = e / W, c = e - rr * W;
      bil_staged<W>(sc, b, rr, c, obuf[e]);
    }
    __syncthreads();  // the stage is read: request the next patch's rows
    if (lp + 1 < p1) stage(lp + 1, st + ((lp + 1 - p0) & 1) * (R + 1) * SP);
    cp_async_commit();
    float2 v[G::N1];
    if (act && lane < G::N2) inv_stepB<W>(v, lane, lbuf);
    __syncthreads();
    if (act && lane < G::N2) {
#pragma unroll
      for (int n1 = 0; n1 < G::N1; ++n1) {
        const int c = G::N2 * n1 + lane;
        const float2 o = obuf[r * W + c];
        const float2 Pk = __ldg(P + ((size_t)k * W + r0 + r) * W + c);
        gp[(k * R + r) * W + c] = cadd(gp[(k * R + r) * W + c], cmulc(v[n1], o));  // conj(o) G_psi
        tbuf[(k * R + r) * W + c] = cmulc(v[n1], Pk);                              // conj(P) G_psi
      }
    }
    __syncthreads();
    float gy = 0.f, gx = 0.f;
    float2* gout = scratch + (((size_t)lp * npl + M) * W + r0) * W;
    for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
      const int rr = e / W, c = e - rr * W;
      float2 g = make_float2(0.f, 0.f);
      for (int kk = 0; kk < M; ++kk) g = cadd(g, tbuf[(kk * R + rr) * W + c]);
      float2 o, dy, dx;
      bil_staged<W>(sc, b, rr, c, o, &dy, &dx);
      gy += g.x * dy.x + g.y * dy.y;  // Re(conj(G_o) do/dy)
      gx += g.x * dx.x + g.y * dx.y;
      gout[(size_t)rr * W + c] = g;
    }
    gy = warp_sum(gy);
    gx = warp_sum(gx);
    if ((threadIdx.x & 31) == 0) {
      gw[((lp - p0) * 8 + (threadIdx.x >> 5)) * 2] = gy;
      gw[((lp - p0) * 8 + (threadIdx.x >> 5)) * 2 + 1] = gx;
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  {
    const int nw = (blockDim.x + 31) >> 5;
    for (int t = threadIdx.x; t < p1 - p0; t += blockDim.x) {
      float sy = 0.f, sx = 0.f;
      for (int w = 0; w < nw; ++w) {  // fixed order
        sy += gw[(t * 8 + w) * 2];
        sx += gw[(t * 8 + w) * 2 + 1];
      }
      gpos_part[((size_t)sj[t] * nrb + blockIdx.x) * 2] = sy;
      gpos_part[((size_t)sj[t] * nrb + blockIdx.x) * 2 + 1] = sx;
    }
  }
  const int slot = blockIdx.y;
  for (int e = threadIdx.x; e < M * R * W; e += blockDim.x) {
    const int kk = e / (R * W), rem = e - kk * R * W, rr = rem / W, c = rem - rr * W;
    const size_t g = (((size_t)slot * M + kk) * W + r0 + rr) * W + c;
    gP_part[g] = accumulate ? cadd(gP_part[g], gp[e]) : gp[e];
  }
}

// ---------------------------------------------------- dL/dO scatter
// Gather form of the bilinear transpose over the (W+1)^2 footprint; the
// footprints of one group are disjoint, so plain read-modify-writes suffice.
template <int W>
__global__ void __launch_bounds__(256)
k_grad_scatter(float2* __restrict__ gO, int Hx, const int* __restrict__ ids,
               const float* __restrict__ pos, const float2* __restrict__ scratch, int npl,
               int M) {
  const int lp = blockIdx.y;
  pdl_trigger();
  pdl_wait();  // G_o comes from the inverse-row pass
  const Bil b = bil_of(pos, ids[lp]);
  const float2* G = scratch + ((size_t)lp * npl + M) * W * W;
  const float w[2][2] = {{(1.f - b.fy) * (1.f - b.fx), (1.f - b.fy) * b.fx},
                         {b.fy * (1.f - b.fx), b.fy * b.fx}};
  const int n = (W + 1) * (W + 1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int p = e / (W + 1), q = e - p * (W + 1);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int rr = p - a, cc = q - c;
        if (rr >= 0 && rr < W && cc >= 0 && cc < W) {
          const float2 g = G[(size_t)rr * W + cc];
          acc.x = fmaf(w[a][c], g.x, acc.x);
          acc.y = fmaf(w[a][c], g.y, acc.y);
        }
      }
    float2* t = gO + (size_t)(b.iy + p) * Hx + b.ix + q;
    *t = cadd(*t, acc);
  }
}

// ---------------------------------------------------- final fixed-order sums
__global__ void k_grad_sum_probe(const float2* __restrict__ part, int nslots, size_t n,
                                 float2* __restrict__ gP) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < nslots; ++k) s = cadd(s, part[(size_t)k * n + i]);
    gP[i] = s;
  }
}
// dL/dpos_j: the row blocks' partial (y, x) pairs of position j, one warp per
// position (coalesced), each lane summing a fixed strided subset in order,
// then a fixed shuffle tree: deterministic.
__global__ void k_grad_sum_pos(const float2* __restrict__ part, int nrb, int N,
                               float* __restrict__ gpos) {
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), l = threadIdx.x & 31;
  if (j >= N) return;  // whole warps
  float sy = 0.f, sx = 0.f;
  for (int b = l; b < nrb; b += 32) {
    const float2 v = part[(size_t)j * nrb + b];
    sy += v.x;
    sx += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  if (l == 0) {
    gpos[2 * j] = sy;
    gpos[2 * j + 1] = sx;
  }
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

static size_t grad_inv_smem(const Tiling& t) {
  int LP = 0;
  switch (t.W) {
    case 32: LP = Line<32>::LP; break;
    case 64: LP = Line<64>::LP; break;
    case 96: LP = Line<96>::LP; break;
    case 128: LP = Line<128>::LP; break;
    case 192: LP = Line<192>::LP; break;
    default: LP = Line<256>::LP; break;
  }
  const int TB = std::max(t.M * t.R * LP, t.M * t.R * t.W);
  return (size_t)(t.W + t.M * t.R * t.W + TB + t.M * t.R * t.W + t.R * t.W +
                  2 * (t.R + 1) * (t.W + 1)) * sizeof(float2) +
         (size_t)t.ppc * (sizeof(Bil) + sizeof(int) + 8 * 2 * sizeof(float));
}

static size_t grad_fwd_smem(const Tiling& t) {
  int LP = 0;
  switch (t.W) {
    case 32: LP = Line<32>::LP; break;
    case 64: LP = Line<64>::LP; break;
    case 96: LP = Line<96>::LP; break;
    case 128: LP = Line<128>::LP; break;
    case 192: LP = Line<192>::LP; break;
    default: LP = Line<256>::LP; break;
  }
  return (size_t)(t.W + t.M * t.R * t.W + t.M * t.R * LP + t.R * t.W +
                  2 * (t.R + 1) * (t.W + 1)) * sizeof(float2) + (size_t)t.ppc * sizeof(Bil);
}

cudaError_t set_grad_smem(const Tiling& t) {
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(t.W, {
    e = allow_max_smem((const void*)k_grad_rows_fwd<WW>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_grad_rows_inv<WW>);
  });
  return e;
}

cudaError_t launch_grad_rows_fwd(const Tiling& t, const float2* O, int Hx, const float2* P,
                                 const int* ids, const float* pos, int npatch,
                                 const float2* tw, float2* scratch, int npl, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppc - 1) / t.ppc);
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(t.W, e = launch_pdl(k_grad_rows_fwd<WW>, grid, dim3(t.thrC), grad_fwd_smem(t),
                                     s, O, Hx, P, t.M, t.R, t.ppc, ids, pos, npatch, tw,
                                     scratch, npl));
  return e;
}

cudaError_t launch_grad_rows_inv(const Tiling& t, const float2* O, int Hx, const float2* P,
                                 const int* ids, const float* pos, int npatch,
                                 float2* scratch, int npl, const float2* tw, float2* gP_part,
                                 int accumulate, float* gpos_part, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppc - 1) / t.ppc);
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(t.W, e = launch_pdl(k_grad_rows_inv<WW>, grid, dim3(t.thrC), grad_inv_smem(t),
                                     s, O, Hx, P, t.M, t.R, t.ppc, ids, pos, npatch, scratch,
                                     npl, tw, gP_part, accumulate, gpos_part));
  return e;
}

cudaError_t launch_grad_scatter(int W, int M, float2* gO, int Hx, const int* ids,
                                const float* pos, int npatch, const float2* scratch, int npl,
                                cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  const int blocks = ((W + 1) * (W + 1) + 255) / 256;
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(W, e = launch_pdl(k_grad_scatter<WW>, dim3(blocks, npatch), dim3(256), 0, s,
                                   gO, Hx, ids, pos, scratch, npl, M));
  return e;
}

cudaError_t launch_grad_finish(const Tiling& t, int nslots, const float2* gP_part, float2* gP,
                               const float* gpos_part, int N, float* gpos,
                               const float* loss_part, size_t nloss, float* loss,
                               double* tmp, cudaStream_t s) {
  const size_t n = (size_t)t.M * t.W * t.W;
  if (gP) k_grad_sum_probe<<<(int)std::min<size_t>(1184, (n + 255) / 256), 256, 0, s>>>(
      gP_part, nslots, n, gP);
  if (gpos)
    k_grad_sum_pos<<<(int)(((size_t)N * 32 + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float2*>(gpos_part), t.W / t.R, N, gpos);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the loss: the same two-level fixed-order double sum as the iteration error
  return launch_err_reduce(loss_part, nloss, 1.0, nullptr, loss, tmp, s);
}

}  // namespace pty
