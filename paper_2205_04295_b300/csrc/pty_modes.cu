// Orthogonalisation of the probe modes (the mixed state of Eq. 4 of Guzzi et
// al., arXiv 2205.04295, after the multimode ePIE of Thibault & Menzel,
// Nature 494, 68, 2013): with the Gram matrix G_kl = sum_r conj(P_k) P_l =
// V diag(lambda) V^H (decreasing lambda), the modes become P'_m = sum_k V_km
// P_k: mutually orthogonal, |P'_m|^2 summed over r equal to lambda_m, the
// density matrix sum_k P_k(r) conj(P_k(r')) unchanged.  Each eigenvector's
// unit phase is fixed by making its largest-magnitude entry (the first on
// ties) real and positive.
//
// k_gram reduces each entry over the W^2 pixels in double precision (fixed
// order: bitwise repeatable); the M x M eigenproblem (M <= 16) is solved on
// the host by cyclic complex Jacobi rotations in double precision; k_mix
// applies V to every pixel in place.
#include "pty_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace pty {

namespace {

__global__ void __launch_bounds__(256)
k_gram(const float2* __restrict__ P, int M, int WW, double2* __restrict__ G) {
  __shared__ double2 red[256];
  const int k = blockIdx.x / M, l = blockIdx.x - k * M;
  const float2* a = P + (size_t)k * WW;
  const float2* b = P + (size_t)l * WW;
  double sr = 0.0, si = 0.0;
  for (int r = threadIdx.x; r < WW; r += blockDim.x) {
    const double ax = a[r].x, ay = a[r].y, bx = b[r].x, by = b[r].y;
    sr += ax * bx + ay * by;  // conj(a) b
    si += ax * by - ay * bx;
  }
  red[threadIdx.x] = make_double2(sr, si);
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) G[blockIdx.x] = red[0];
}

// P'_m(r) = sum_k V[k][m] P_k(r), in place (one pixel per thread, M <= 16).
__global__ void __launch_bounds__(256)
k_mix(float2* __restrict__ P, int M, int WW, const float2* __restrict__ V) {
  __shared__ float2 v[16 * 16];
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) v[e] = V[e];
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < WW; r += gridDim.x * blockDim.x) {
    float2 p[16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < M) p[k] = P[(size_t)k * WW + r];
    for (int m = 0; m < M; ++m) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < M) {
          const float2 a = v[k * M + m], b = p[k];
          acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
          acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
        }
      P[(size_t)m * WW + r] = acc;
    }
  }
}

}  // namespace

// Cyclic Jacobi for a Hermitian matrix: each rotation first turns the pivot
// A_pq = r e^{i phi} real (column q times e^{-i phi}), then zeroes it by the
// real rotation with tan(theta) = t, t = sgn(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (A_qq - A_pp) / (2 r).  Eigenvalues in decreasing order (stable),
// eigenvector phases fixed as in the header.
int hermitian_eig(int M, const std::complex<double>* A_in, double* w,
                  std::complex<double>* V_out) {
  using C = std::complex<double>;
  if (M < 1 || M > 16) return -1;
  std::vector<C> A(A_in, A_in + (size_t)M * M), V((size_t)M * M, C(0.0));
  for (int i = 0; i < M; ++i) V[(size_t)i * M + i] = 1.0;
  auto at = [&](std::vector<C>& X, int i, int j) -> C& { return X[(size_t)i * M + j]; };
  double scale = 0.0;
  for (int i = 0; i < M; ++i) scale += std::norm(at(A, i, i));
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < M; ++p)
      for (int q = p + 1; q < M; ++q) off += std::norm(at(A, p, q));
    if (off <= 1e-30 * scale || off == 0.0) break;
    for (int p = 0; p < M; ++p)
      for (int q = p + 1; q < M; ++q) {
        const C apq = at(A, p, q);
        const double r = std::abs(apq);
        if (r == 0.0) continue;
        const C ph = apq / r;  // e^{i phi}
        const double tau = (at(A, q, q).real() - at(A, p, p).real()) / (2.0 * r);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        const C e = std::conj(ph);  // e^{-i phi}
        // A <- A U, V <- V U: columns p, q
        for (int i = 0; i < M; ++i) {
          const C x = at(A, i, p), y = at(A, i, q);
          at(A, i, p) = c * x - s * e * y;
          at(A, i, q) = s * x + c * e * y;
          const C vx = at(V, i, p), vy = at(V, i, q);
          at(V, i, p) = c * vx - s * e * vy;
          at(V, i, q) = s * vx + c * e * vy;
        }
        // A <- U^H A: rows p, q
        for (int j = 0; j < M; ++j) {
          const C x = at(A, p, j), y = at(A, q, j);
          at(A, p, j) = c * x - s * ph * y;
          at(A, q, j) = s * x + c * ph * y;
        }
        at(A, p, q) = at(A, q, p) = 0.0;
        at(A, p, p) = at(A, p, p).real();
        at(A, q, q) = at(A, q, q).real();
      }
  }
  // decreasing eigenvalues (stable), phases fixed
  std::vector<int> ord(M);
  for (int i = 0; i < M; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int a, int b) { return at(A, a, a).real() > at(A, b, b).real(); });
  for (int m = 0; m < M; ++m) {
    const int src = ord[m];
    w[m] = at(A, src, src).real();
    int imax = 0;
    double best = -1.0;
    for (int i = 0; i < M; ++i) {
      const double a = std::abs(at(V, i, src));
      if (a > best) {
        best = a;
        imax = i;
      }
    }
    const C fix = best > 0 ? std::conj(at(V, imax, src)) / best : C(1.0);
    for (int i = 0; i < M; ++i) V_out[(size_t)i * M + m] = at(V, i, src) * fix;
  }
  return 0;
}

cudaError_t launch_gram(const float2* P, int M, int WW, void* G, cudaStream_t s) {
  k_gram<<<M * M, 256, 0, s>>>(P, M, WW, static_cast<double2*>(G));
  return cudaGetLastError();
}

cudaError_t launch_mix(float2* P, int M, int WW, const float2* V, cudaStream_t s) {
  k_mix<<<std::min(1184, (WW + 255) / 256), 256, 0, s>>>(P, M, WW, V);
  return cudaGetLastError();
}

}  // namespace pty
