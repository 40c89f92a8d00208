// M-rPIE group step on sm_103a: the kernels of the three passes over one
// chunk of a group of pairwise-disjoint crop boxes, the probe update at the
// end of the group, small reductions, the line-FFT utilities and the host
// launchers (bodies in pty_passes.cuh).
#include "pty_passes.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdint>

namespace pty {

namespace {

template <int W>
__global__ void __launch_bounds__(256, 4)
k_rows_fwd(const float2* __restrict__ O, int Hx, const float2* __restrict__ P,
           int M, int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           const float2* __restrict__ tw_g, float2* __restrict__ scratch,
           float* __restrict__ omax_part, int npl, int xo) {
  rows_fwd_body<W, false>(O, Hx, P, M, R, ppc, ids, corners, npatch, tw_g, scratch, omax_part, npl,
                          xo, blockIdx.x, blockIdx.y);
}

// Two CTAs per SM.  BIG launches up to 384 threads and holds 80 registers a
// thread; the others launch at most 320 threads (M * CB * lanes <= 320, e.g.
// 5 modes x 4 columns x 16 lanes) and may hold 96, which removes the spills
// of the 80-register build (22.2 -> 21.4 ms per iteration at 256², 5 modes).
// With use_tma the far-field block is staged by TMA through `tmap` (a
// time-out sets *err).
constexpr int kColsSmall = 320;  // threads of the 96-register column kernels
template <int W, int CB, bool GRAD, bool BIG>
__global__ void __launch_bounds__(BIG ? 384 : kColsSmall, 2)
k_cols(float2* __restrict__ scratch, int M,
       const uint16_t* __restrict__ I, const int* __restrict__ ids,
       const float2* __restrict__ tw_g, float inv_w, float eps,
       float* __restrict__ err_part, int npl, int ppcb, int npatch,
       const __grid_constant__ CUtensorMap tmap, int use_tma, int* err, int xb, int plane0) {
  // Patch blocks in reverse order: CTAs are dispatched in blockIdx order, so
  // this pass starts on the patches pass A wrote last and pass C (forward)
  // starts on the ones this pass writes last.  A group's far field is larger
  // than L2 at big W and M; in one direction every pass would miss on all of
  // it (least-recently-used eviction of a stream larger than the cache).
  // Each patch's outputs are the same in any order.
  cols_body<W, CB, GRAD>(scratch, M, I, ids, tw_g, inv_w, eps, err_part, npl, ppcb, npatch,
                         blockIdx.x, gridDim.y - 1 - blockIdx.y, use_tma ? &tmap : nullptr, err,
                         xb, plane0);
}

template <int W, bool PSTAGE>
__global__ void __launch_bounds__(256, 2)
k_rows_inv(float2* __restrict__ O, int Hx, const float2* __restrict__ P, int M,
           int R, int ppc, const int* __restrict__ ids,
           const int2* __restrict__ corners, int npatch,
           float2* __restrict__ scratch, const float* __restrict__ omax_part,
           const float* __restrict__ pmax_part, int n_pmax,
           const float2* __restrict__ tw_g, UpdArgs a,
           float2* __restrict__ pnum, float* __restrict__ pden,
           float* __restrict__ osum, int accumulate, int npl, int refine, int* err) {
  rows_inv_body<W, false, PSTAGE>(O, Hx, P, M, R, ppc, ids, corners, npatch, scratch, omax_part,
                                  pmax_part, n_pmax, tw_g, a, pnum, pden, osum, accumulate, npl,
                                  refine, blockIdx.x, blockIdx.y, err);
}

__global__ void __launch_bounds__(256)
k_probe_apply(float2* __restrict__ P, int M, int WW, const float2* __restrict__ pnum,
              const float* __restrict__ pden, const float* __restrict__ osum,
              int nslots, float alpha_P, float reg_eps, float* __restrict__ pmax_part) {
  probe_apply_body(P, M, WW, pnum, pden, osum, nslots, alpha_P, reg_eps, pmax_part, blockIdx.x, gridDim.x);
}

// Probe update of the per-pass path, one thread per (pixel, mode): block
// (kPaX pixels, M modes), grid n_pmax blocks of WW / n_pmax pixels each.  A
// thread's slot sums (denominator and its mode's numerator, slot order)
// load eight slots at a time, both sums' loads in flight together; the new
// probe intensity sum_k |P_k|^2 of a pixel is added in mode order through
// shared memory and the block's maximum goes to pmax_part[block].  The same
// arithmetic as probe_apply_body, which the batched form keeps.
constexpr int kPaX = 128;
__global__ void __launch_bounds__(1024)
k_probe_apply_pm(float2* __restrict__ P, int M, int WW, const float2* __restrict__ pnum,
                 const float* __restrict__ pden, const float* __restrict__ osum, int nslots,
                 float alpha_P, float reg_eps, float* __restrict__ pmax_part) {
  __shared__ float pint_s[8][kPaX];
  __shared__ float red[32];
  pdl_trigger();
  pdl_wait();
  const int x = threadIdx.x, k = threadIdx.y;
  float os = 0.f;
  for (int s = 0; s < nslots; ++s) os += osum[s];
  const float guard = reg_eps * os;
  const int ppb = (WW + gridDim.x - 1) / gridDim.x;  // pixels of this block
  float lmax = 0.f;
  constexpr int kB = 8;
  for (int i0 = 0; i0 < ppb; i0 += kPaX) {
    const int pix = blockIdx.x * ppb + i0 + x;
    const bool on = i0 + x < ppb && pix < WW;
    if (on) {
      float d = 0.f;
      float2 n = make_float2(0.f, 0.f);
      for (int s0 = 0; s0 < nslots; s0 += kB) {
        float dv[kB];
        float2 nv[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const bool in = s0 + u < nslots;
          dv[u] = in ? pden[(size_t)(s0 + u) * WW + pix] : 0.f;
          nv[u] = in ? pnum[((size_t)(s0 + u) * M + k) * WW + pix] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          if (s0 + u < nslots) {
            d += dv[u];
            n = cadd(n, nv[u]);
          }
        }
      }
      const float dd = d + guard;
      const float sc = dd > 0.f ? alpha_P / dd : 0.f;  // zero numerator too
      float2 p = P[(size_t)k * WW + pix];
      p = make_float2(fmaf(sc, n.x, p.x), fmaf(sc, n.y, p.y));
      P[(size_t)k * WW + pix] = p;
      pint_s[k][x] = cabs2(p);
    }
    __syncthreads();
    if (on && k == 0) {
      float pint = 0.f;
      for (int kk = 0; kk < M; ++kk) pint += pint_s[kk][x];
      lmax = fmaxf(lmax, pint);
    }
    __syncthreads();
  }
  // the mode-0 threads are the first kPaX / 32 warps (linear index x + kPaX k)
  if (k == 0) {
    const float m = warp_max(lmax);
    if ((x & 31) == 0) red[x >> 5] = m;
  }
  __syncthreads();
  if (x == 0 && k == 0) {
    float m = 0.f;
    for (int i = 0; i < kPaX / 32; ++i) m = fmaxf(m, red[i]);
    pmax_part[blockIdx.x] = m;
  }
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

// The iteration's error: kErrParts CTAs each sum a fixed contiguous range of
// the per-(pattern, column block) partials in double (fixed order), then one
// CTA sums their kErrParts results in order and normalises.  Deterministic;
// one CTA over all 10^4 x 64 partials took 0.38 ms per iteration.
constexpr int kErrParts = kErrPartsMax;
__global__ void __launch_bounds__(256)
k_err_partial(const float* __restrict__ part, size_t n, double* __restrict__ out) {
  __shared__ double red[256];
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t b0 = (size_t)blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
  double s = 0.0;
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += (double)part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256)
k_err_reduce(const double* __restrict__ part, size_t n, double inv_sumI,
             const unsigned long long* sum_dev, float* out) {
  err_reduce_body(part, n, inv_sumI, sum_dev, out);
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
    sincospi(-2.0 * tw_exponent(W, e) / W, &sn, &cs);
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
    sincospi(-2.0 * tw_exponent(W, e) / W, &sn, &cs);
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

int smem_per_sm() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return 228 * 1024;
  }
  return v;
}

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
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem_optin() - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  // prefer the largest shared-memory carveout: otherwise the driver may pick
  // one that holds a single CTA of the larger tilings per SM
  return cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
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

bool encode_far_field_map(const void* base, int W, size_t planes, int CB, CUtensorMap* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // TMA rules: 16-byte aligned base, strides multiples of 16 bytes, box inner
  // extent (CB complex = 8 CB bytes) a multiple of 16, every box extent <= 256
  if (!base || reinterpret_cast<uintptr_t>(base) % 16 || CB < 2 || CB % 2 || CB > 256 ||
      W > 256 || planes < 1 || planes > (1ull << 32))
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)W, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)W * sizeof(float2), (cuuint64_t)W * W * sizeof(float2)};
  const cuuint32_t box[3] = {(cuuint32_t)CB, (cuuint32_t)W, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return encode(out, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void*>(base), dims, strides,
                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tiling_fits(const Tiling& t) {
  const size_t lim = (size_t)smem_optin() - 1024;
  return t.thrA <= 256 && t.thrB <= 384 && t.thrC <= 256 && t.smA_staged <= lim && t.smB <= lim &&
         t.smC <= lim;
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

// Column-block widths the column pass is compiled for.
#define PTY_DISPATCH_CB(CB, ...)                      \
  switch (CB) {                                       \
    case 2: { constexpr int CBB = 2; __VA_ARGS__; } break; \
    case 4: { constexpr int CBB = 4; __VA_ARGS__; } break; \
    case 8: { constexpr int CBB = 8; __VA_ARGS__; } break; \
    case 16: { constexpr int CBB = 16; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;            \
  }

// Pass C may copy its probe rows to shared memory only where that costs it no
// CTA per SM: the occupancy of k_rows_inv<W> at thr threads with sm0 and with
// sm1 bytes of dynamic shared memory (false if it cannot be queried).
bool pstage_pays(int W, int thr, size_t sm0, size_t sm1) {
  const void *f0 = nullptr, *f1 = nullptr;
  switch (W) {
    case 32: f0 = (const void*)k_rows_inv<32, false>; f1 = (const void*)k_rows_inv<32, true>; break;
    case 64: f0 = (const void*)k_rows_inv<64, false>; f1 = (const void*)k_rows_inv<64, true>; break;
    case 96: f0 = (const void*)k_rows_inv<96, false>; f1 = (const void*)k_rows_inv<96, true>; break;
    case 128: f0 = (const void*)k_rows_inv<128, false>; f1 = (const void*)k_rows_inv<128, true>; break;
    case 192: f0 = (const void*)k_rows_inv<192, false>; f1 = (const void*)k_rows_inv<192, true>; break;
    case 256: f0 = (const void*)k_rows_inv<256, false>; f1 = (const void*)k_rows_inv<256, true>; break;
    default: return false;
  }
  int n0 = 0, n1 = 0;
  if (allow_max_smem(f0) != cudaSuccess || allow_max_smem(f1) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, f0, thr, sm0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, f1, thr, sm1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n1 > 0 && n1 >= n0;
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
  t.ppcc = t.ppc;
  t.ppcb = 2;
  int CB = pow2_floor(std::max(1, max_threads_b / (M * L)));
  CB = std::max(2, std::min(16, CB));  // M * CB * L <= max_threads_b threads
  while ((W / 2) % CB) CB /= 2;
  if (CB_req > 0) CB = CB_req;
  t.CB = CB;
  t.thrA = round32(MA * R * L);
  t.thrC = round32(M * R * L);
  t.thrB = round32(M * CB * L);
  // the per-pass kernel reads its probe rows through L1; the batched form's
  // task function stages them (smA_staged)
  t.smA = (size_t)(W + MA * R * LP + 2 * R * W + t.ppc) * sizeof(float2);
  t.smA_staged = t.smA + (size_t)M * R * W * sizeof(float2);
  // pass B transforms the M modes only (the crop plane's column DFTs are
  // taken by the registration's correlation pass)
  t.smB = (size_t)(W + M * W * CB + M * CB * LP) * sizeof(float2) +
          (size_t)M * CB * W * sizeof(float) + (size_t)2 * W * CB * sizeof(uint16_t) +
          (size_t)64 * sizeof(int) +  // pattern ids of up to 64 patches per CTA
          128;                        // alignment of the stage
  t.smI = (size_t)(W + M * CB * LP) * sizeof(float2) + (size_t)M * CB * W * sizeof(float);
  const int TB = std::max(M * R * LP, M * R * W);
  const size_t smC0 = (size_t)(W + TB + 2 * R * W + M * R * W) *
                          sizeof(float2) +
                      (size_t)2 * R * W * sizeof(float) + (size_t)t.ppc * (sizeof(int2) + sizeof(float));
  const size_t smC1 = smC0 + (size_t)M * R * W * sizeof(float2);
  t.pstage = pstage_pays(W, t.thrC, smC0, smC1) ? 1 : 0;
  t.smC = t.pstage ? smC1 : smC0;
  // probe-update blocks (and probe-intensity maxima): one per 256 pixels, or
  // one per 128 where that would leave SMs idle (W <= 192; at 128^2 / 3
  // modes, 137 groups: 4.34 -> 4.00 ms per iteration)
  t.n_pmax = W * W / 256 < 148 ? W * W / 128 : W * W / 256;
  t.n_pmax = std::max(1, std::min(1024, t.n_pmax));
  return t;
}

void fill_residency(Tiling& t) {
  int dev = 0, nsm = 0;
  t.resA = t.resB = t.resC = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const void *fa = nullptr, *fb = nullptr, *fc = nullptr;
  const bool big = t.thrB > kColsSmall;
  auto pick = [&](auto wtag) {
    constexpr int WW = decltype(wtag)::value;
    fa = (const void*)k_rows_fwd<WW>;
    fc = t.pstage ? (const void*)k_rows_inv<WW, true> : (const void*)k_rows_inv<WW, false>;
    switch (t.CB) {
      case 2: fb = big ? (const void*)k_cols<WW, 2, false, true> : (const void*)k_cols<WW, 2, false, false>; break;
      case 4: fb = big ? (const void*)k_cols<WW, 4, false, true> : (const void*)k_cols<WW, 4, false, false>; break;
      case 8: fb = big ? (const void*)k_cols<WW, 8, false, true> : (const void*)k_cols<WW, 8, false, false>; break;
      default: fb = big ? (const void*)k_cols<WW, 16, false, true> : (const void*)k_cols<WW, 16, false, false>; break;
    }
  };
  switch (t.W) {
    case 32: pick(std::integral_constant<int, 32>{}); break;
    case 64: pick(std::integral_constant<int, 64>{}); break;
    case 96: pick(std::integral_constant<int, 96>{}); break;
    case 128: pick(std::integral_constant<int, 128>{}); break;
    case 192: pick(std::integral_constant<int, 192>{}); break;
    default: pick(std::integral_constant<int, 256>{}); break;
  }
  int na = 0, nb = 0, nc = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&na, fa, t.thrA, t.smA) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fb, t.thrB, t.smB) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nc, fc, t.thrC, t.smC) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  t.resA = na * nsm;
  t.resB = nb * nsm;
  t.resC = nc * nsm;
}

namespace {
// Patches per CTA for a kernel whose chunk of n patches makes bx CTAs per
// patch group of q: the q in [lo, hi] that minimises whole waves x (q + a
// CTA's fixed cost of about 3/4 of a patch), the tuned q0 on ties.
int pick_per_cta(int n, int bx, int res, int q0, int lo, int hi) {
  if (res <= 0 || n <= 0) return q0;
  auto cost = [&](int q) {
    const long long ctas = (long long)((n + q - 1) / q) * bx;
    return (double)((ctas + res - 1) / res) * (q + 0.75);
  };
  int best = q0;
  double bc = cost(q0);
  for (int q = lo; q <= hi; ++q) {
    const double c = cost(q);
    if (c < bc - 1e-9 || (c < bc + 1e-9 && std::abs(q - q0) < std::abs(best - q0))) {
      best = q;
      bc = c;
    }
  }
  return best;
}
}  // namespace

Tiling tiling_for_chunk(const Tiling& t, int n) {
  Tiling c = t;
  const int qa = pick_per_cta(n, t.W / t.R, t.resA, t.ppc, std::max(1, t.ppc / 2),
                              std::min(64, 2 * t.ppc));
  c.ppcb = pick_per_cta(n, t.W / t.CB, t.resB, t.ppcb, 1, std::min(64, 2 * t.ppcb + 1));
  // pass A's corner list is ppc long
  c.smA = t.smA + ((size_t)qa - t.ppc) * sizeof(float2);
  c.smA_staged = t.smA_staged + ((size_t)qa - t.ppc) * sizeof(float2);
  c.ppc = qa;
  return c;
}

cudaError_t set_smem_limits(const Tiling& t) {
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(t.W, {
    e = allow_max_smem((const void*)k_rows_fwd<WW>);
    for (int cb = 2; cb <= 16 && e == cudaSuccess; cb *= 2) {
      PTY_DISPATCH_CB(cb, {
        e = allow_max_smem((const void*)k_cols<WW, CBB, false, false>);
        if (e == cudaSuccess) e = allow_max_smem((const void*)k_cols<WW, CBB, true, false>);
        if (e == cudaSuccess) e = allow_max_smem((const void*)k_cols<WW, CBB, false, true>);
        if (e == cudaSuccess) e = allow_max_smem((const void*)k_cols<WW, CBB, true, true>);
      });
    }
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_rows_inv<WW, false>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_rows_inv<WW, true>);
    if (e == cudaSuccess)
      e = allow_max_smem((const void*)k_cols_intensity<WW>);
  });
  return e;
}

void make_twiddles(int W, float2* out) {
  const double pi = 3.14159265358979323846;
  for (int e = 0; e < W; ++e) {
    const double th = -2.0 * pi * (double)tw_exponent(W, e) / (double)W;
    out[e] = make_float2((float)std::cos(th), (float)std::sin(th));
  }
}

cudaError_t launch_rows_fwd(const Tiling& t, const float2* O, int Hx, const float2* P,
                            const int* ids, const int2* corners, int npatch,
                            const float2* tw, float2* scratch, float* omax_part,
                            cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppc - 1) / t.ppc);
  cudaError_t e = cudaSuccess;
  PTY_DISPATCH_W(t.W, e = launch_pdl(k_rows_fwd<WW>, grid, dim3(t.thrA), t.smA, s, O, Hx, P,
                                     t.M, t.R, t.ppc, ids, corners, npatch, tw, scratch,
                                     omax_part, t.npl, t.xo));
  return e;
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
                        float eps, float* err_part, const CUtensorMap* tm, int* err,
                        cudaStream_t s, int xb, int plane0) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.CB, (npatch + t.ppcb - 1) / t.ppcb);
  cudaError_t e = cudaSuccess;
  CUtensorMap none{};
  const bool big = t.thrB > kColsSmall;
  PTY_DISPATCH_W(t.W, PTY_DISPATCH_CB(t.CB, e = big ? launch_pdl(k_cols<WW, CBB, false, true>,
                                                           grid, dim3(t.thrB), t.smB, s, scratch,
                                                           t.M, I, ids, tw, inv_w, eps, err_part,
                                                           t.npl, t.ppcb, npatch,
                                                           tm ? *tm : none, tm ? 1 : 0, err, xb, plane0)
                                                    : launch_pdl(k_cols<WW, CBB, false, false>,
                                                           grid, dim3(t.thrB), t.smB, s, scratch,
                                                           t.M, I, ids, tw, inv_w, eps, err_part,
                                                           t.npl, t.ppcb, npatch,
                                                           tm ? *tm : none, tm ? 1 : 0, err, xb, plane0)));
  return e;
}

cudaError_t launch_cols_grad(const Tiling& t, float2* scratch, const uint16_t* I,
                             const int* ids, int npatch, const float2* tw, float inv_w,
                             float delta, float* loss_part, int npl, const CUtensorMap* tm,
                             int* err, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.CB, (npatch + t.ppcb - 1) / t.ppcb);
  cudaError_t e = cudaSuccess;
  CUtensorMap none{};
  const bool big = t.thrB > kColsSmall;
  PTY_DISPATCH_W(t.W, PTY_DISPATCH_CB(t.CB, e = big ? launch_pdl(k_cols<WW, CBB, true, true>,
                                                           grid, dim3(t.thrB), t.smB, s, scratch,
                                                           t.M, I, ids, tw, inv_w, delta,
                                                           loss_part, npl, t.ppcb, npatch,
                                                           tm ? *tm : none, tm ? 1 : 0, err, -1, 0)
                                                    : launch_pdl(k_cols<WW, CBB, true, false>,
                                                           grid, dim3(t.thrB), t.smB, s, scratch,
                                                           t.M, I, ids, tw, inv_w, delta,
                                                           loss_part, npl, t.ppcb, npatch,
                                                           tm ? *tm : none, tm ? 1 : 0, err, -1, 0)));
  return e;
}

cudaError_t launch_rows_inv(const Tiling& t, float2* O, int Hx, const float2* P,
                            const int* ids, const int2* corners, int npatch,
                            float2* scratch, const float* omax_part,
                            const float* pmax_part, const float2* tw,
                            const UpdArgs& a, float2* pnum, float* pden,
                            float* osum, int accumulate, int* err, cudaStream_t s,
                            int refine) {
  if (npatch <= 0) return cudaSuccess;
  dim3 grid(t.W / t.R, (npatch + t.ppcc - 1) / t.ppcc);
  cudaError_t e = cudaSuccess;
  const int rf = refine < 0 ? t.refine : (refine && t.refine);
  PTY_DISPATCH_W(t.W, e = t.pstage
      ? launch_pdl(k_rows_inv<WW, true>, grid, dim3(t.thrC), t.smC, s, O, Hx, P, t.M, t.R, t.ppcc,
                   ids, corners, npatch, scratch, omax_part, pmax_part, t.n_pmax, tw, a, pnum,
                   pden, osum, accumulate, t.npl, rf, err)
      : launch_pdl(k_rows_inv<WW, false>, grid, dim3(t.thrC), t.smC, s, O, Hx, P, t.M, t.R,
                   t.ppcc, ids, corners, npatch, scratch, omax_part, pmax_part, t.n_pmax, tw, a,
                   pnum, pden, osum, accumulate, t.npl, rf, err));
  return e;
}

cudaError_t launch_probe_apply(const Tiling& t, float2* P, const float2* pnum,
                               const float* pden, const float* osum, int nslots,
                               float alpha_P, float reg_eps, float* pmax_part,
                               cudaStream_t s) {
  if (t.M >= 2 && t.M <= 8)  // one mode: the per-pixel kernel has twice the threads a block
    return launch_pdl(k_probe_apply_pm, dim3(t.n_pmax), dim3(kPaX, t.M), 0, s, P, t.M,
                      t.W * t.W, pnum, pden, osum, nslots, alpha_P, reg_eps, pmax_part);
  return launch_pdl(k_probe_apply, dim3(t.n_pmax), dim3(256), 0, s, P, t.M, t.W * t.W, pnum,
                    pden, osum, nslots, alpha_P, reg_eps, pmax_part);
}

cudaError_t launch_pmax(const Tiling& t, const float2* P, float* pmax_part, cudaStream_t s) {
  k_pmax<<<t.n_pmax, 256, 0, s>>>(P, t.M, t.W * t.W, pmax_part);
  return cudaGetLastError();
}

cudaError_t launch_err_reduce(const float* err_part, size_t n, double inv_sumI,
                              const unsigned long long* sum_dev, float* out, double* tmp,
                              cudaStream_t s) {
  k_err_partial<<<kErrParts, 256, 0, s>>>(err_part, n, tmp);
  k_err_reduce<<<1, 256, 256 * sizeof(double), s>>>(tmp, kErrParts, inv_sumI, sum_dev, out);
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

}  // namespace pty
