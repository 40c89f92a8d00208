// Model intensities without any allocation: pty_model_intensities_noalloc.
//
// Who needs this: code that may not call cudaMalloc at all -- for example a
// caller running inside another framework's memory pool that forbids foreign
// allocations, a real-time loop that must never hit the allocator's
// implicit device synchronisation, or an embedded host that reserves all
// device memory up front.  Such a caller cannot create a pty_handle (which
// owns its buffers), so this entry point takes every input and output as a
// caller-owned device pointer and keeps its only intermediate, the far-field
// rows of a few patches, in the fixed array below.
//
// The array is a file-scope __device__ variable of PTY_NOALLOC_SCRATCH_BYTES:
// every GPU that loads the library holds it until the process exits.  All
// calls share it, so calls that overlap on the GPU (on different streams,
// from different threads) race and must be serialised by the caller.  Each
// call writes every scratch element before reading it, so nothing in it has
// to start at zero.
//
// Host code never dereferences the array's symbol (on the host it is only a
// stand-in, not a device address): every call resolves the device address
// with cudaGetSymbolAddress in the context current at the call and passes it
// to the kernels.  The lookup allocates nothing and costs about a
// microsecond; it is not cached, because an address belongs to the module as
// loaded in one context, and a cache keyed on the device number would go
// stale after cudaDeviceReset or under a caller's own (non-primary) driver
// context on the same device.  The first call in a context may make the
// runtime load the library's module there, so it should come before any
// stream capture.
#include "pty_fft.cuh"
#include "pty_internal.h"
#include "../../include/pty.h"

namespace {

constexpr size_t kScratchElems = PTY_NOALLOC_SCRATCH_BYTES / sizeof(float2);
static __device__ __align__(256) float2 g_noalloc_scratch[kScratchElems];

int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

// Crop corner floor(p + 0.5) and whether the W x W box lies inside the object.
__device__ __forceinline__ bool na_corner(const float* pos, int j, int W, int Hy, int Hx,
                                          int& cy, int& cx) {
  const float y = pos[2 * j], x = pos[2 * j + 1];
  if (!isfinite(y) || !isfinite(x)) return false;
  cy = (int)floorf(y);
  cx = (int)floorf(x);
  if (y - (float)cy >= 0.5f) ++cy;
  if (x - (float)cx >= 0.5f) ++cx;
  return cy >= 0 && cx >= 0 && cy + W <= Hy && cx + W <= Hx;
}

__device__ void na_twiddles(float2* tw, int W) {
  for (int e = threadIdx.x; e < W; e += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * pty::tw_exponent(W, e) / W, &sn, &cs);
    tw[e] = make_float2((float)cs, (float)sn);
  }
}

// Rows: psi_p = P_p o_j for each mode, forward row DFTs into the scratch.
template <int W>
__global__ void __launch_bounds__(256)
k_na_rows(const float2* __restrict__ O, int Hy, int Hx, const float2* __restrict__ P, int M,
          int R, const float* __restrict__ pos, int j0, float2* __restrict__ scratch) {
  using G = pty::Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  na_twiddles(tw, W);
  __syncthreads();
  const int lp = blockIdx.y, r0 = blockIdx.x * R;
  int cy = 0, cx = 0;
  const bool inside = na_corner(pos, j0 + lp, W, Hy, Hx, cy, cx);
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < M * R;
  const int k = act ? line / R : 0, r = act ? line - k * R : 0;
  float2* lbuf = tbuf + line * G::LP;
  if (act && lane < G::N2) {
    float2 v[G::N1];
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) {
      const int c = G::N2 * n1 + lane;
      v[n1] = inside ? pty::cmul(P[((size_t)k * W + r0 + r) * W + c],
                                 O[(size_t)(cy + r0 + r) * Hx + cx + c])
                     : make_float2(0.f, 0.f);
    }
    pty::fwd_step1<W>(v, lane, tw, lbuf);
  }
  __syncthreads();
  if (act && lane < G::N1) {
    float2 z[G::N2];
    pty::fwd_step3<W>(z, lane, lbuf);
    float2* dst = scratch + (((size_t)lp * M + k) * W + r0 + r) * W;
#pragma unroll
    for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = z[k2];
  }
}

// Columns: forward column DFTs, S = sum_p |Psi_p|^2 written detector-centred.
// A pattern whose crop box leaves the object is written as NaN.
template <int W>
__global__ void __launch_bounds__(512)
k_na_cols(const float2* __restrict__ scratch, int Hy, int Hx, int M, int CB,
          const float* __restrict__ pos, int j0, float* __restrict__ out) {
  using G = pty::Line<W>;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* tbuf = tw + W;
  float* Sb = reinterpret_cast<float*>(tbuf + M * CB * G::LP);
  na_twiddles(tw, W);
  const int lp = blockIdx.y, c0 = blockIdx.x * CB;
  const int c = threadIdx.x % CB, rest = threadIdx.x / CB;
  const int lane = rest % G::L, k = rest / G::L;
  const bool act = k < M;
  const float2* col = scratch + ((size_t)lp * M + (act ? k : 0)) * W * W + c0 + c;
  float2* lbuf = tbuf + ((act ? k : 0) * CB + c) * G::LP;
  __syncthreads();
  if (act && lane < G::N2) {
    float2 v[G::N1];
#pragma unroll
    for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = col[(size_t)(G::N2 * n1 + lane) * W];
    pty::fwd_step1<W>(v, lane, tw, lbuf);
  }
  __syncthreads();
  if (act && lane < G::N1) {
    float2 z[G::N2];
    pty::fwd_step3<W>(z, lane, lbuf);
#pragma unroll
    for (int k2 = 0; k2 < G::N2; ++k2) Sb[(k * CB + c) * W + lane + G::N1 * k2] = pty::cabs2(z[k2]);
  }
  __syncthreads();
  int cy, cx;
  const bool inside = na_corner(pos, j0 + lp, W, Hy, Hx, cy, cx);
  const float f2 = 1.0f / ((float)W * (float)W);
  for (int e = threadIdx.x; e < CB * W; e += blockDim.x) {
    const int u = e / CB, cl = e - u * CB;
    float s = 0.f;
    for (int kk = 0; kk < M; ++kk) s += Sb[(kk * CB + cl) * W + u];
    const int iu = (u + W / 2) % W, iv = (c0 + cl + W / 2) % W;
    out[((size_t)(j0 + lp) * W + iu) * W + iv] = inside ? s * f2 : __int_as_float(0x7fc00000);
  }
}

struct NaShape {
  int R, CB, thrR, thrC;
  size_t smR, smC;
};

template <int W> NaShape na_shape(int M) {
  using G = pty::Line<W>;
  NaShape s{};
  int R = pow2_floor(256 / (M * G::L) > 0 ? 256 / (M * G::L) : 1);
  if (R > 16) R = 16;
  while (W % R) R /= 2;
  int CB = pow2_floor(512 / (M * G::L) > 0 ? 512 / (M * G::L) : 1);
  CB = CB < 2 ? 2 : (CB > 16 ? 16 : CB);
  while ((W / 2) % CB) CB /= 2;
  s.R = R;
  s.CB = CB;
  s.thrR = (M * R * G::L + 31) / 32 * 32;
  s.thrC = (M * CB * G::L + 31) / 32 * 32;
  s.smR = (size_t)(W + M * R * G::LP) * sizeof(float2);
  s.smC = (size_t)(W + M * CB * G::LP) * sizeof(float2) + (size_t)M * CB * W * sizeof(float);
  return s;
}

template <int W>
cudaError_t na_run(const float2* O, int Hy, int Hx, const float2* P, int M, const float* pos,
                   int N, float* out, float2* scratch, cudaStream_t st) {
  const NaShape s = na_shape<W>(M);
  cudaError_t e = cudaFuncSetAttribute(k_na_rows<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)s.smR);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_na_cols<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smC);
  if (e != cudaSuccess) return e;
  const size_t per_patch = (size_t)M * W * W;
  const int chunk = (int)(kScratchElems / per_patch);
  for (int j0 = 0; j0 < N; j0 += chunk) {
    const int n = N - j0 < chunk ? N - j0 : chunk;
    k_na_rows<W><<<dim3(W / s.R, n), s.thrR, s.smR, st>>>(O, Hy, Hx, P, M, s.R, pos, j0, scratch);
    k_na_cols<W><<<dim3(W / s.CB, n), s.thrC, s.smC, st>>>(scratch, Hy, Hx, M, s.CB, pos, j0, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" int pty_model_intensities_noalloc(const void* O, int Hy, int Hx, const void* P,
                                             int M, int W, const float* pos, int N, float* out,
                                             void* stream) {
  if (!O || !P || !pos || !out) return pty::set_error(PTY_EINVAL, "null pointer");
  if (!pty::supported_W(W)) return pty::set_error(PTY_EINVAL, "unsupported pattern size W=%d", W);
  if (M < 1 || M > 16) return pty::set_error(PTY_EINVAL, "M=%d outside 1..16", M);
  if (N < 1 || Hy < W || Hx < W) return pty::set_error(PTY_EINVAL, "bad N or object size");
  const size_t need = (size_t)M * W * W * sizeof(float2);
  if (need > PTY_NOALLOC_SCRATCH_BYTES)
    return pty::set_error(PTY_EINVAL,
                          "one %dx%d pattern with %d modes needs %zu bytes of far-field scratch; "
                          "the fixed no-allocation scratch holds %zu",
                          W, W, M, need, (size_t)PTY_NOALLOC_SCRATCH_BYTES);
  // the address in the context current now (see the top of this file)
  void* addr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
  if (e != cudaSuccess || !addr)
    return pty::set_error(PTY_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  float2* scratch = static_cast<float2*>(addr);
  const float2* Oc = static_cast<const float2*>(O);
  const float2* Pc = static_cast<const float2*>(P);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (W) {
    case 32: e = na_run<32>(Oc, Hy, Hx, Pc, M, pos, N, out, scratch, st); break;
    case 64: e = na_run<64>(Oc, Hy, Hx, Pc, M, pos, N, out, scratch, st); break;
    case 96: e = na_run<96>(Oc, Hy, Hx, Pc, M, pos, N, out, scratch, st); break;
    case 128: e = na_run<128>(Oc, Hy, Hx, Pc, M, pos, N, out, scratch, st); break;
    case 192: e = na_run<192>(Oc, Hy, Hx, Pc, M, pos, N, out, scratch, st); break;
    default: e = na_run<256>(Oc, Hy, Hx, Pc, M, pos, N, out, scratch, st); break;
  }
  if (e != cudaSuccess) return pty::set_error(PTY_ECUDA, "launch: %s", cudaGetErrorString(e));
  return PTY_OK;
}
