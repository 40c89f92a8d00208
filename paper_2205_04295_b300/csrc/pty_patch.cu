// Fused single-kernel M-rPIE patch path for patterns up to 128 x 128 (the
// M-rPIE section of Guzzi et al., arXiv 2205.04295: exit waves Eq. 1 and 4,
// unitary far-field DFT Eq. 2, mixed-state modulus constraint Eq. 7, object
// update Eq. 6 and the probe update's sums Eq. 5).
//
// One thread-block cluster of M x S CTAs works on one patch at a time; CTA
// (mode k, slab s) keeps rows [s W/S, (s+1) W/S) of mode k's W x W plane in
// shared memory for the whole patch:
//
//   forward row DFTs of psi_k = P_k o_j on the slab's rows        (local)
//   forward column DFTs over the S slabs of mode k, in place      (DSMEM)
//   constraint: S = sum_k |Psi_k|^2, Psi_k *= sqrt(I)/(sqrt(S)+eps) on this
//   CTA's share of the slab's pixels, for every mode              (DSMEM)
//   inverse column DFTs, in place                                 (DSMEM)
//   inverse row DFTs                                              (local)
//   object update and probe sums on this CTA's share of the pixels,
//   summing D_k conj(P_k) over the modes                          (DSMEM)
//
// so that a patch reads its crop, probe rows and counts and writes its crop
// and probe sums once, with no far-field scratch (the registration's crop
// planes excepted).  Every step repeats the three-pass path's arithmetic
// (the same line DFTs, constraint and update expressions and summation
// orders over the modes); the probe sums are grouped per cluster instead of
// per CTA column.
//
// A CTA's share of a slab is the rows lr = k, k + M, ... of the slab (whole
// rows, so that with XCORR_A it can also row-transform its rows of the
// refined crop).  The cluster barrier separates the six phases; a CTA never
// reads another's slab outside the phase that owns it, and the last barrier
// keeps every CTA resident until no other one reads its slab.
#include "pty_cluster.cuh"
#include "pty_passes.cuh"

#include <algorithm>

namespace pty {

namespace {

constexpr int kPatchMaxThreads = 512;

template <int W, int S>
__host__ __device__ constexpr bool patch_ok() {
  return W <= 128 && W % S == 0 && (W / S) % Line<W>::N1 == 0 && (W / S) % Line<W>::N2 == 0;
}

template <int W, int S>
__global__ void __launch_bounds__(kPatchMaxThreads, 1) k_patch(const __grid_constant__ PatchArgs q) {
  using G = Line<W>;
  constexpr int HS = W / S;     // rows (and columns) of the slab
  constexpr int PITCH = W + 1;  // odd row pitch: a column line's lanes hit distinct banks
  static_assert(patch_ok<W, S>(), "a slab holds whole DFT sub-blocks of a column line");
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* A = tw + W;                    // HS x PITCH: this CTA's slab
  float2* lbase = A + HS * PITCH;        // NL transpose lines
  __shared__ float red_o[32], red_e[32];
  __shared__ float xch[2];               // read by the cluster: [0] crop maximum, [1] error
  __shared__ float s_pmax;

  const int M = q.M, NL = q.NL;
  const int CS = M * S;
  const int rank = (int)cluster_rank();
  const int k = rank / S, s = rank - k * S;
  const int cid = blockIdx.x / CS, ncl = gridDim.x / CS;
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < NL;
  float2* lbuf = lbase + (act ? line : 0) * G::LP;
  const int r0 = s * HS;  // first row of the slab; also the first column of its column lines
  const int nw = blockDim.x >> 5;
  const int nown = (HS - k + M - 1) / M;  // slab rows lr = k, k + M, ... this CTA owns
  float2* Am[S];                          // mode k's slabs
#pragma unroll
  for (int t = 0; t < S; ++t) Am[t] = cluster_map(A, (unsigned)(k * S + t));

  pdl_trigger();
  for (int e = threadIdx.x; e < W; e += blockDim.x) tw[e] = q.tw[e];
  pdl_wait();  // O, P and the probe maxima come from the previous kernels
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int i = threadIdx.x; i < q.n_pmax; i += 32) m = fmaxf(m, q.pmax_part[i]);
    m = warp_max(m);
    if (threadIdx.x == 0) s_pmax = m;
  }
  __syncthreads();
  const float pmax = s_pmax;
  const float gden = fmaf(q.a.gamma, pmax, q.a.reg_eps * pmax);
  float osum_local = 0.f;
  bool first = true;

  for (int lp = cid; lp < q.npatch; lp += ncl) {
    const int j = q.ids[lp];
    const int2 cc = q.corners[j];
    if (!first) cluster_sync();  // the previous patch's remote reads of the slabs are over

    // ---- forward row DFTs of psi_k = P_k o_j; with XCORR_A also this CTA's
    // rows of the crop itself (registration plane M)
    const int nlines = HS + (q.refine == 1 ? nown : 0);
    float omax = 0.f;
    for (int t0 = 0; t0 < nlines; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < nlines;
      const bool crop = t >= HS;
      const int lr = crop ? k + M * (t - HS) : t;
      if (on && lane < G::N2) {
        const float2* orow = q.O + (size_t)(cc.x + r0 + lr) * q.Hx + cc.y;
        const float2* prow = q.P + ((size_t)k * W + r0 + lr) * W;
        float2 v[G::N1];
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) {
          const int c = G::N2 * n1 + lane;
          const float2 o = orow[c];
          v[n1] = crop ? o : cmul(__ldg(prow + c), o);
          omax = fmaxf(omax, cabs2(o));
        }
        fwd_step1<W>(v, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N1) {
        float2 z[G::N2];
        fwd_step3<W>(z, lane, lbuf);
        float2* dst = crop ? q.scratch + (((size_t)lp * q.npl + M) * W + r0 + lr) * W
                           : A + lr * PITCH;
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = z[k2];
      }
      line_sync<W>();
    }
    omax = warp_max(omax);
    if ((threadIdx.x & 31) == 0) red_o[threadIdx.x >> 5] = omax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
      for (int i = 0; i < nw; ++i) m = fmaxf(m, red_o[i]);
      xch[0] = m;
    }
    cluster_sync();  // rows transformed; each slab's crop maximum posted
    float om = 0.f;  // max_r |o_j(r)|^2 over the whole crop (exact: a maximum)
#pragma unroll
    for (int t = 0; t < S; ++t) om = fmaxf(om, *cluster_map(&xch[0], (unsigned)(k * S + t)));

    // ---- forward column DFTs of mode k, columns [r0, r0 + HS), in place
    for (int t0 = 0; t0 < HS; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < HS;
      const int c = r0 + t;
      if (on && lane < G::N2) {
        float2 v[G::N1];
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) {
          const int ow = (G::N2 * n1) / HS;  // a constant once unrolled
          v[n1] = Am[ow][(G::N2 * n1 - ow * HS + lane) * PITCH + c];
        }
        fwd_step1<W>(v, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N1) {
        float2 z[G::N2];
        fwd_step3<W>(z, lane, lbuf);
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) {
          const int ow = (G::N1 * k2) / HS;
          Am[ow][(G::N1 * k2 - ow * HS + lane) * PITCH + c] = z[k2];
        }
      }
      line_sync<W>();
    }
    cluster_sync();  // Psi_k complete in every slab

    // ---- modulus constraint on this CTA's rows of slab s, every mode (the
    // three-pass column kernel's arithmetic, in the same order)
    float e_acc = 0.f;
    {
      const float f2 = q.inv_w * q.inv_w;
      const uint16_t* Ij = q.I + (size_t)j * W * W;
      for (int e = threadIdx.x; e < nown * W; e += blockDim.x) {
        const int rw = e / W, c = e - rw * W;
        const int lr = k + M * rw, u = r0 + lr, off = lr * PITCH + c;
        const float cnt = (float)__ldg(Ij + (size_t)((u + W / 2) % W) * W + (c + W / 2) % W);
        float2 z[8];
        float sum = 0.f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          if (jj < M) {
            z[jj] = cluster_map(A, (unsigned)(jj * S + s))[off];
            sum += cabs2(z[jj]);
          }
        }
        const float sI = sqrt_rs(cnt);
        const float a = __fmul_rn(sqrt_rs(sum), q.inv_w);
        const float d = __fsub_rn(a, sI);
        e_acc = fmaf(d, d, e_acc);
        const float f = __fmul_rn(__fdividef(sI, __fadd_rn(a, q.a.eps)), f2);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (jj < M) cluster_map(A, (unsigned)(jj * S + s))[off] = cscale(z[jj], f);
        if (q.refine == 2) {
          // XCORR_B: model intensity and counts, unshifted, as real parts of
          // registration planes M and M + 1
          float2* pl = q.scratch + ((size_t)lp * q.npl + M) * W * W + (size_t)u * W + c;
          pl[0] = make_float2(sum * f2, 0.f);
          pl[(size_t)W * W] = make_float2(cnt, 0.f);
        }
      }
    }
    e_acc = warp_sum(e_acc);
    if ((threadIdx.x & 31) == 0) red_e[threadIdx.x >> 5] = e_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int i = 0; i < nw; ++i) t += red_e[i];  // fixed order
      xch[1] = t;
    }
    cluster_sync();  // every mode scaled; every CTA's error partial posted
    if (rank == 0 && threadIdx.x == 0) {
      float t = 0.f;
      for (int r = 0; r < CS; ++r) t += *cluster_map(&xch[1], (unsigned)r);  // rank order
      float* ep = q.err_part + (size_t)j * q.nb;
      ep[0] = t;
      for (int i = 1; i < q.nb; ++i) ep[i] = 0.f;
    }

    // ---- inverse column DFTs, in place
    for (int t0 = 0; t0 < HS; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < HS;
      const int c = r0 + t;
      if (on && lane < G::N1) {
        float2 z[G::N2];
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) {
          const int ow = (G::N1 * k2) / HS;
          z[k2] = Am[ow][(G::N1 * k2 - ow * HS + lane) * PITCH + c];
        }
        inv_stepA<W>(z, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N2) {
        float2 v[G::N1];
        inv_stepB<W>(v, lane, lbuf);
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) {
          const int ow = (G::N2 * n1) / HS;
          Am[ow][(G::N2 * n1 - ow * HS + lane) * PITCH + c] = v[n1];
        }
      }
      line_sync<W>();
    }
    cluster_sync();

    // ---- inverse row DFTs of the slab: psi'_k (unnormalised by W^2, which
    // the constraint factor carries)
    for (int t0 = 0; t0 < HS; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < HS;
      if (on && lane < G::N1) {
        float2 z[G::N2];
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = A[t * PITCH + lane + G::N1 * k2];
        inv_stepA<W>(z, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N2) {
        float2 v[G::N1];
        inv_stepB<W>(v, lane, lbuf);
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) A[t * PITCH + G::N2 * n1 + lane] = v[n1];
      }
      line_sync<W>();
    }
    cluster_sync();  // psi'_k complete in every slab

    // ---- object update (written in place: the group's boxes are disjoint)
    // and the probe sums of this cluster's slot, on this CTA's rows
    {
      const bool acc = !first || q.accumulate;
      const float omb = 1.f - q.a.beta, omg = 1.f - q.a.gamma, bom = q.a.beta * om;
      const int slot = cid;
      for (int e = threadIdx.x; e < nown * W; e += blockDim.x) {
        const int rw = e / W, c = e - rw * W;
        const int lr = k + M * rw, r = r0 + lr, off = lr * PITCH + c;
        float2* op = q.O + (size_t)(cc.x + r) * q.Hx + cc.y + c;
        float* pd = q.pden + ((size_t)slot * W + r) * W + c;
        const float2 o = *op;
        const float pd0 = acc ? *pd : 0.f;
        float2 pv[8], vv[8], nv[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          if (jj < M) {
            pv[jj] = __ldg(q.P + ((size_t)jj * W + r) * W + c);
            vv[jj] = cluster_map(A, (unsigned)(jj * S + s))[off];
            nv[jj] = acc ? q.pnum[(((size_t)slot * M + jj) * W + r) * W + c] : make_float2(0.f, 0.f);
          }
        }
        float2 sT = make_float2(0.f, 0.f);
        float pint = 0.f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          if (jj < M) {
            const float2 D = csub(vv[jj], cmul(pv[jj], o));
            sT = cadd(sT, cmulc(D, pv[jj]));
            pint += cabs2(pv[jj]);
            const float2 nm = cmulc(D, o);
            nv[jj] = acc ? cadd(nv[jj], nm) : nm;
          }
        }
        const float dn = fmaf(omg, pint, gden);
        const float sc = dn > 0.f ? q.a.alpha_O / dn : 0.f;  // a zero denominator has a zero numerator
        const float2 onw = make_float2(fmaf(sc, sT.x, o.x), fmaf(sc, sT.y, o.y));
        *op = onw;
        if (q.refine == 1) A[off] = onw;  // only this CTA reads its own rows
        const float dv = fmaf(omb, cabs2(o), bom);
        *pd = acc ? pd0 + dv : dv;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (jj < M) q.pnum[(((size_t)slot * M + jj) * W + r) * W + c] = nv[jj];
      }
      osum_local += om;
    }

    // ---- XCORR_A: forward row DFTs of this CTA's rows of the refined crop
    // (registration plane M + 1)
    if (q.refine == 1) {
      __syncthreads();
      for (int t0 = 0; t0 < nown; t0 += NL) {
        const int t = t0 + line;
        const bool on = act && t < nown;
        const int lr = k + M * t;
        if (on && lane < G::N2) {
          float2 v[G::N1];
#pragma unroll
          for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = A[lr * PITCH + G::N2 * n1 + lane];
          fwd_step1<W>(v, lane, tw, lbuf);
        }
        line_sync<W>();
        if (on && lane < G::N1) {
          float2 z[G::N2];
          fwd_step3<W>(z, lane, lbuf);
          float2* dst = q.scratch + (((size_t)lp * q.npl + M + 1) * W + r0 + lr) * W;
#pragma unroll
          for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = z[k2];
        }
        line_sync<W>();
      }
    }
    first = false;
  }
  cluster_sync();  // no CTA leaves while another may still read its slab
  if (rank == 0 && threadIdx.x == 0 && !first)
    q.osum[cid] = q.accumulate ? q.osum[cid] + osum_local : osum_local;
}

template <int W, int S>
void* patch_fn() {
  if constexpr (patch_ok<W, S>())
    return reinterpret_cast<void*>(k_patch<W, S>);
  else
    return nullptr;
}

template <int W>
void* patch_fn_w(int S) {
  switch (S) {
    case 1: return patch_fn<W, 1>();
    case 2: return patch_fn<W, 2>();
    case 4: return patch_fn<W, 4>();
    case 8: return patch_fn<W, 8>();
    default: return nullptr;
  }
}

void* patch_kernel(int W, int S) {
  switch (W) {
    case 32: return patch_fn_w<32>(S);
    case 64: return patch_fn_w<64>(S);
    case 96: return patch_fn_w<96>(S);
    case 128: return patch_fn_w<128>(S);
    default: return nullptr;
  }
}

template <int W> void patch_line(int& L, int& LP) {
  L = Line<W>::L;
  LP = Line<W>::LP;
}

}  // namespace

cudaError_t set_patch_smem(int W) {
  cudaError_t e = cudaSuccess;
  for (int S = 1; S <= 8 && e == cudaSuccess; S *= 2)
    if (void* f = patch_kernel(W, S)) e = allow_max_smem(f);
  return e;
}

PatchGeo make_patch_geo(int W, int M, int S) {
  PatchGeo g = {};
  g.W = W;
  g.M = M;
  g.S = S;
  void* f = patch_kernel(W, S);
  if (!f || M < 1 || M * S > 8) return g;
  int L = 16, LP = 0;
  switch (W) {
    case 32: patch_line<32>(L, LP); break;
    case 64: patch_line<64>(L, LP); break;
    case 96: patch_line<96>(L, LP); break;
    default: patch_line<128>(L, LP); break;
  }
  const int HS = W / S;
  if (HS < M) return g;  // every CTA of a slab owns at least one row
  g.NL = std::min(HS, 32);
  g.NT = (g.NL * L + 31) / 32 * 32;
  if (g.NT > kPatchMaxThreads) return g;
  g.sm = (size_t)(W + HS * (W + 1) + g.NL * LP) * sizeof(float2);
  if (g.sm > (size_t)smem_optin() - 512) return g;
  if (allow_max_smem(f) != cudaSuccess) {
    cudaGetLastError();
    return g;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(M * S);
  cfg.blockDim = dim3(g.NT);
  cfg.dynamicSmemBytes = g.sm;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = M * S;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  g.ncap = n;
  return g;
}

cudaError_t launch_patch(const PatchGeo& g, const PatchArgs& a, int nclusters, cudaStream_t s) {
  void* f = patch_kernel(g.W, g.S);
  if (!f || g.ncap < 1 || nclusters < 1 || nclusters > g.ncap || a.M != g.M)
    return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * g.M * g.S);
  cfg.blockDim = dim3(g.NT);
  cfg.dynamicSmemBytes = g.sm;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g.M * g.S;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  PatchArgs q = a;
  q.NL = g.NL;
  return cudaLaunchKernelEx(&cfg, reinterpret_cast<void (*)(PatchArgs)>(f), q);
}

}  // namespace pty
