// Register-resident small DFTs and the two steps of a length-W line FFT.
//
// A length-W DFT is split as W = N1 * N2 (the "four-step" factorisation):
//
//   X[k1 + N1 k2] = sum_n2 w_N2^{n2 k2} w_W^{n2 k1} sum_n1 x[N2 n1 + n2] w_N1^{n1 k1}
//
// forward step 1: lane n2 (< N2) holds x[N2 n1 + n2], n1 = 0..N1-1, takes a
//                 DFT_N1 and multiplies by the twiddles w_W^{n2 k1};
// shared-memory transpose;
// forward step 3: lane k1 (< N1) holds the N2 values of row k1, takes a
//                 DFT_N2 and so ends with X[k1 + N1 k2], k2 = 0..N2-1.
//
// The inverse runs the same two steps backwards (DFT_N2 with conjugate
// twiddles, transpose, DFT_N1), taking the frequency-ordered values a lane
// holds after forward step 3 and returning the natural-ordered samples a lane
// held before forward step 1.  Nothing is normalised here; callers scale.
//
// Twiddles w_W^m = exp(-2 pi i m / W) come from a table of W entries computed
// in double precision and rounded to float.  Slot e holds w_W^m with
// m = tw_exponent(W, e): for a square factorisation (N1 = N2 = N) slot a N + b
// holds w^{a b}, so that both steps read lane-consecutive slots (step 1 reads
// w^{lane k1} at k1 N + lane, inverse step A w^{n2 lane} at n2 N + lane: no
// shared-memory bank conflicts); otherwise slot m holds w^m.  The constants
// inside the small DFTs (cos/sin of multiples of pi/8 and pi/6) are written
// out below.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PTY_D __device__ __forceinline__

namespace pty {

PTY_D float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
PTY_D float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
PTY_D float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
PTY_D float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
PTY_D float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
PTY_D float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// multiply by -i (forward) or +i (inverse)
template <bool INV> PTY_D float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by exp(-i t) (forward) or exp(+i t) (inverse), c = cos t, s = sin t
// (the fused multiply-adds are written out, so that every kernel rounds the
// same way whatever the compiler would contract)
template <bool INV> PTY_D float2 rot(float2 a, float c, float s) {
  return INV ? make_float2(fmaf(a.x, c, -(a.y * s)), fmaf(a.x, s, a.y * c))
             : make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -(a.x * s)));
}
// multiply by table twiddle w (forward) or conj(w) (inverse)
template <bool INV> PTY_D float2 twiddle(float2 a, float2 w) {
  return INV ? cmulc(a, w) : cmul(a, w);
}

constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f;  // sin(pi/8)
constexpr float kS3 = 0.86602540378443864676f;   // sin(pi/3)

template <int N, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
  static PTY_D void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV> struct Dft<3, INV> {
  static PTY_D void run(float2* v) {
    float2 t = cadd(v[1], v[2]);
    float2 m = make_float2(fmaf(-0.5f, t.x, v[0].x), fmaf(-0.5f, t.y, v[0].y));
    float2 r = mul_mi<INV>(csub(v[1], v[2]));
    v[0] = cadd(v[0], t);
    v[1] = make_float2(fmaf(kS3, r.x, m.x), fmaf(kS3, r.y, m.y));
    v[2] = make_float2(fmaf(-kS3, r.x, m.x), fmaf(-kS3, r.y, m.y));
  }
};

template <bool INV> struct Dft<4, INV> {
  static PTY_D void run(float2* v) {
    float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    float2 c = cadd(v[1], v[3]), d = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

// 8 = 2 x 4, decimation in time
template <bool INV> struct Dft<8, INV> {
  static PTY_D void run(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    o[1] = rot<INV>(o[1], kC8, kC8);
    o[2] = mul_mi<INV>(o[2]);
    o[3] = rot<INV>(o[3], -kC8, kC8);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

// 16 = 4 x 4: DFT_4 over m of x[r + 4m], twiddle w16^{r q}, DFT_4 over r
template <bool INV> struct Dft<16, INV> {
  static PTY_D void run(float2* v) {
    float2 y[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int m = 0; m < 4; ++m) y[r][m] = v[r + 4 * m];
      Dft<4, INV>::run(y[r]);
    }
    // twiddles w16^{rq}: rq in {1,2,3,4,6,9}
    y[1][1] = rot<INV>(y[1][1], kC16, kS16);
    y[1][2] = rot<INV>(y[1][2], kC8, kC8);
    y[1][3] = rot<INV>(y[1][3], kS16, kC16);
    y[2][1] = rot<INV>(y[2][1], kC8, kC8);
    y[2][2] = mul_mi<INV>(y[2][2]);
    y[2][3] = rot<INV>(y[2][3], -kC8, kC8);
    y[3][1] = rot<INV>(y[3][1], kS16, kC16);
    y[3][2] = rot<INV>(y[3][2], -kC8, kC8);
    y[3][3] = rot<INV>(y[3][3], -kC16, -kS16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 z[4] = {y[0][q], y[1][q], y[2][q], y[3][q]};
      Dft<4, INV>::run(z);
#pragma unroll
      for (int p = 0; p < 4; ++p) v[q + 4 * p] = z[p];
    }
  }
};

// 12 = 3 x 4 by the prime-factor (Good-Thomas) map: input n = (4 n1 + 3 n2)
// mod 12, output k = (4 k1 + 9 k2) mod 12 with k1 = k mod 3, k2 = k mod 4.
template <bool INV> struct Dft<12, INV> {
  static PTY_D void run(float2* v) {
    float2 a[3][4];
#pragma unroll
    for (int n1 = 0; n1 < 3; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < 4; ++n2) a[n1][n2] = v[(4 * n1 + 3 * n2) % 12];
      Dft<4, INV>::run(a[n1]);
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      float2 b[3] = {a[0][k2], a[1][k2], a[2][k2]};
      Dft<3, INV>::run(b);
#pragma unroll
      for (int k1 = 0; k1 < 3; ++k1) v[(4 * k1 + 9 * k2) % 12] = b[k1];
    }
  }
};

// N of a square factorisation W = N x N (0 if the factors differ).
__host__ __device__ constexpr int tw_square(int W) { return W == 256 ? 16 : W == 64 ? 8 : 0; }
// Exponent m of the twiddle w_W^m held in table slot e (0 <= e < W).
__host__ __device__ constexpr int tw_exponent(int W, int e) {
  return tw_square(W) ? (e / tw_square(W)) * (e % tw_square(W)) : e;
}

// Factorisation per supported pattern size.
template <int W> struct Geo;
template <> struct Geo<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Geo<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Geo<96> { static constexpr int N1 = 8, N2 = 12; };
template <> struct Geo<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Geo<192> { static constexpr int N1 = 16, N2 = 12; };
template <> struct Geo<256> { static constexpr int N1 = 16, N2 = 16; };

template <int W> struct Line {
  static constexpr int N1 = Geo<W>::N1;
  static constexpr int N2 = Geo<W>::N2;
  static constexpr int L = N1 > N2 ? N1 : N2;  // lanes per line
  // transpose buffer: one pad element after every N2 elements, and a line
  // pitch = 4 (mod 16) elements so that lines differ in bank.
  static constexpr int RAW = W + W / N2;
  static constexpr int LP = RAW + ((20 - (RAW % 16)) % 16);
  static PTY_D int sp(int s) { return s + s / N2; }
  static constexpr bool SQ = N1 == N2;
  static_assert(tw_square(W) == (SQ ? N1 : 0), "twiddle layout and factorisation disagree");
  // table slot of w^{lane k1} (forward step 1, lane = n2) and of w^{n2 lane}
  // (inverse step A, lane = k1)
  static PTY_D int twf(int k1, int lane) { return SQ ? k1 * N2 + lane : lane * k1; }
  static PTY_D int twi(int n2, int lane) { return SQ ? n2 * N1 + lane : n2 * lane; }
};

// ---- forward step 1: v[n1] = x[N2 n1 + lane] on entry (lane < N2); leaves
// the twiddled DFT_N1 outputs in the transpose buffer line `buf`.
template <int W>
PTY_D void fwd_step1(float2* v, int lane, const float2* tw, float2* buf) {
  using G = Line<W>;
  __builtin_assume(lane >= 0 && lane < G::N2);  // lets the padded offsets fold to constants
  Dft<G::N1, false>::run(v);
#pragma unroll
  for (int k1 = 0; k1 < G::N1; ++k1) {
    float2 t = k1 ? cmul(v[k1], tw[G::twf(k1, lane)]) : v[k1];
    buf[G::sp(G::N2 * k1 + lane)] = t;
  }
}

// ---- forward step 3 (lane < N1): z[k2] = X[lane + N1 k2] on exit.
template <int W>
PTY_D void fwd_step3(float2* z, int lane, const float2* buf) {
  using G = Line<W>;
  __builtin_assume(lane >= 0 && lane < G::N1);
#pragma unroll
  for (int n2 = 0; n2 < G::N2; ++n2) z[n2] = buf[G::sp(G::N2 * lane + n2)];
  Dft<G::N2, false>::run(z);
}

// ---- inverse step A (lane < N1): z[k2] = X[lane + N1 k2] on entry.
template <int W>
PTY_D void inv_stepA(float2* z, int lane, const float2* tw, float2* buf) {
  using G = Line<W>;
  __builtin_assume(lane >= 0 && lane < G::N1);
  Dft<G::N2, true>::run(z);
#pragma unroll
  for (int n2 = 0; n2 < G::N2; ++n2) {
    float2 t = n2 ? cmulc(z[n2], tw[G::twi(n2, lane)]) : z[n2];
    buf[G::sp(G::N2 * lane + n2)] = t;
  }
}

// ---- inverse step B (lane < N2): v[n1] = x[N2 n1 + lane] (unnormalised) on exit.
template <int W>
PTY_D void inv_stepB(float2* v, int lane, const float2* buf) {
  using G = Line<W>;
  __builtin_assume(lane >= 0 && lane < G::N2);
#pragma unroll
  for (int k1 = 0; k1 < G::N1; ++k1) v[k1] = buf[G::sp(G::N2 * k1 + lane)];
  Dft<G::N1, true>::run(v);
}

}  // namespace pty
