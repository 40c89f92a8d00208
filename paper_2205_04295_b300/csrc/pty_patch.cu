// Fused single-kernel M-rPIE patch path for patterns up to 128 x 128 (the
// M-rPIE section of Guzzi et al., arXiv 2205.04295: exit waves Eq. 1 and 4,
// unitary far-field DFT Eq. 2, mixed-state modulus constraint Eq. 7, object
// update Eq. 6 and the probe update's sums Eq. 5).
//
// One thread-block cluster of S CTAs works on one patch at a time.  CTA s
// holds, for every mode, rows [s H, (s+1) H) of the W x W plane (H = W / S,
// "row slab" RA) and, between the two transposes, columns [s H, (s+1) H)
// ("column slab" CA, stored one column line per row of the buffer):
//
//   forward row DFTs of psi_k = P_k o_j on the row slab           (local)
//   gather: column slab from the S row slabs                      (DSMEM)
//   forward column DFTs, modulus constraint S = sum_k |Psi_k|^2,
//   Psi_k *= sqrt(I)/(sqrt(S)+eps), inverse column DFTs           (local)
//   scatter: column slab back into the S row slabs                (DSMEM)
//   inverse row DFTs, object update and probe sums                (local)
//
// Distributed shared memory moves about 15-20 bytes per clock per SM on
// this part (a few times less than L2), so the only cross-CTA traffic is the
// two transposes, 2 (S-1)/S of the patch's far field per CTA, read and
// written in row segments; the sums over the modes never leave a CTA.  A
// patch reads its crop, probe rows and counts and writes its crop and probe
// sums once, with no far-field scratch (the registration's crop planes
// excepted).  Every step repeats the three-pass path's arithmetic (the same
// line DFTs, constraint and update expressions and summation orders over
// the modes); the probe sums are grouped per cluster instead of per CTA
// column.
//
// Ordering: a CTA's row slab is read by the others only between the first
// and the second cluster barrier of a patch (gather) and written by them
// only between the second and the third (scatter); everything else is
// local.  A patch's probe rows and counts are requested (cp.async) as soon as
// its corner is known and used after the forward DFTs.
#include "pty_cluster.cuh"
#include "pty_passes.cuh"

#include <algorithm>

namespace pty {

namespace {

constexpr int kPatchMaxThreads = 512;

template <int W, int S>
__host__ __device__ constexpr bool patch_ok() {
  return W <= 128 && W % S == 0 && (W / S) % 8 == 0;  // 16-byte count pieces
}

template <int W, int S>
__global__ void __launch_bounds__(kPatchMaxThreads, 1) k_patch(const __grid_constant__ PatchArgs q) {
  using G = Line<W>;
  constexpr int H = W / S;      // rows of the row slab, columns of the column slab
  constexpr int PITCH = W + 1;  // odd line pitch: strided accesses hit distinct banks
  static_assert(patch_ok<W, S>(), "slab width");
  const int M = q.M, NL = q.NL;
  extern __shared__ float4 smem4[];
  float2* tw = reinterpret_cast<float2*>(smem4);
  float2* RA = tw + W;                   // [k][r][c]: M x H lines of PITCH
  float2* CA = RA + M * H * PITCH;       // [k][cl][u]: M x H column lines of PITCH
  float2* lbase = CA + M * H * PITCH;    // NL transpose lines
  float2* obuf = lbase + NL * G::LP;     // H x W: the crop rows (then the refined ones)
  float2* pbuf = obuf + H * W;           // M x H x W: the probe rows
  uint16_t* cbuf = reinterpret_cast<uint16_t*>(pbuf + M * H * W);  // W x H counts [u][cl]
  __shared__ float red_o[32], red_e[32];
  __shared__ float xch[2];               // read by the cluster: [0] crop maximum, [1] error
  __shared__ float s_pmax;

  const int s = (int)cluster_rank();
  const int cid = blockIdx.x / S, ncl = gridDim.x / S;
  const int line = threadIdx.x / G::L, lane = threadIdx.x - line * G::L;
  const bool act = line < NL;
  float2* lbuf = lbase + (act ? line : 0) * G::LP;
  const int r0 = s * H;  // first row of the row slab, first column of the column slab
  const int nw = blockDim.x >> 5;
  const int nfar = M * W * H;  // far-field values of one slab (either kind)

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
    {
      // requested now, used after the forward DFTs: every mode's probe rows of
      // the row slab (for the update) and the counts of the column slab
      // (stored fftshifted: row (u + W/2) mod W, columns (c + W/2) mod W;
      // 16-byte pieces that never wrap)
      for (int i = threadIdx.x; i < M * H * (W / 2); i += blockDim.x) {
        const int row = i / (W / 2), h = i - row * (W / 2);  // row = k * H + r
        const int k = row / H, r = row - k * H;
        cp_async<16>(pbuf + row * W + 2 * h, q.P + ((size_t)k * W + r0 + r) * W + 2 * h);
      }
      const uint16_t* Ij = q.I + (size_t)j * W * W;
      constexpr int ppr = H / 8;
      for (int i = threadIdx.x; i < W * ppr; i += blockDim.x) {
        const int u = i / ppr, h = i - u * ppr;
        const int su = (u + W / 2) % W, sc = (r0 + 8 * h + W / 2) % W;
        cp_async<16>(cbuf + u * H + 8 * h, Ij + (size_t)su * W + sc);
      }
      cp_async_commit();
    }

    // ---- forward row DFTs of psi_k = P_k o_j on the row slab; with XCORR_A
    // also the crop rows themselves (registration plane M)
    const int nrl = M * H + (q.refine == 1 ? H : 0);
    float omax = 0.f;
    for (int t0 = 0; t0 < nrl; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < nrl;
      const bool crop = t >= M * H;
      const int k = crop ? M : t / H, r = t - k * H;
      if (on && lane < G::N2) {
        const float2* orow = q.O + (size_t)(cc.x + r0 + r) * q.Hx + cc.y;
        const float2* prow = q.P + ((size_t)(crop ? 0 : k) * W + r0 + r) * W;
        float2 v[G::N1];
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) {
          const int c = G::N2 * n1 + lane;
          const float2 o = orow[c];
          if (k == 0) obuf[r * W + c] = o;
          v[n1] = crop ? o : cmul(__ldg(prow + c), o);
          omax = fmaxf(omax, cabs2(o));
        }
        fwd_step1<W>(v, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N1) {
        float2 z[G::N2];
        fwd_step3<W>(z, lane, lbuf);
        float2* dst = crop ? q.scratch + (((size_t)lp * q.npl + M) * W + r0 + r) * W
                           : RA + (k * H + r) * PITCH;
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
    cluster_sync();  // B1: every row slab transformed; every slab's crop maximum posted
    float om = 0.f;  // max_r |o_j(r)|^2 over the whole crop (exact: a maximum)
#pragma unroll
    for (int t = 0; t < S; ++t) om = fmaxf(om, *cluster_map(&xch[0], (unsigned)t));

    // ---- gather the column slab: CA[k][cl][u] = RA of CTA u / H, [k][u mod H][r0 + cl]
    // (consecutive threads read consecutive columns of one row; four loads in flight)
    for (int e0 = threadIdx.x; e0 < nfar; e0 += 4 * blockDim.x) {
      float2 v[4];
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int e = e0 + q4 * blockDim.x;
        if (e < nfar) {
          const int k = e / (W * H), rem = e - k * (W * H), u = rem / H, cl = rem - u * H;
          const int ow = u / H;
          v[q4] = cluster_map(RA, (unsigned)ow)[(k * H + u - ow * H) * PITCH + r0 + cl];
        }
      }
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int e = e0 + q4 * blockDim.x;
        if (e < nfar) {
          const int k = e / (W * H), rem = e - k * (W * H), u = rem / H, cl = rem - u * H;
          CA[(k * H + cl) * PITCH + u] = v[q4];
        }
      }
    }
    __syncthreads();

    // ---- forward column DFTs (local, in place)
    for (int t0 = 0; t0 < M * H; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < M * H;
      float2* col = CA + t * PITCH;  // column line t = k * H + cl
      if (on && lane < G::N2) {
        float2 v[G::N1];
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = col[G::N2 * n1 + lane];
        fwd_step1<W>(v, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N1) {
        float2 z[G::N2];
        fwd_step3<W>(z, lane, lbuf);
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) col[lane + G::N1 * k2] = z[k2];
      }
      line_sync<W>();
    }
    cp_async_wait<0>();  // this thread's probe and count pieces (the barrier shows all)
    __syncthreads();

    // ---- modulus constraint on the column slab (the three-pass column
    // kernel's arithmetic, in the same order over the modes)
    float e_acc = 0.f;
    {
      const float f2 = q.inv_w * q.inv_w;
      for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
        const int u = e / H, cl = e - u * H;
        const float cnt = (float)cbuf[e];
        float sum = 0.f;
        for (int k = 0; k < M; ++k) sum += cabs2(CA[(k * H + cl) * PITCH + u]);
        const float sI = sqrt_rs(cnt);
        const float a = __fmul_rn(sqrt_rs(sum), q.inv_w);
        const float d = __fsub_rn(a, sI);
        e_acc = fmaf(d, d, e_acc);
        const float f = __fmul_rn(__fdividef(sI, __fadd_rn(a, q.a.eps)), f2);
        for (int k = 0; k < M; ++k) {
          float2* z = CA + (k * H + cl) * PITCH + u;
          *z = cscale(*z, f);
        }
        if (q.refine == 2) {
          // XCORR_B: model intensity and counts, unshifted, as real parts of
          // registration planes M and M + 1
          float2* pl = q.scratch + ((size_t)lp * q.npl + M) * W * W + (size_t)u * W + r0 + cl;
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

    // ---- inverse column DFTs (local, in place)
    for (int t0 = 0; t0 < M * H; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < M * H;
      float2* col = CA + t * PITCH;
      if (on && lane < G::N1) {
        float2 z[G::N2];
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = col[lane + G::N1 * k2];
        inv_stepA<W>(z, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N2) {
        float2 v[G::N1];
        inv_stepB<W>(v, lane, lbuf);
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) col[G::N2 * n1 + lane] = v[n1];
      }
      line_sync<W>();
    }
    cluster_sync();  // B2: every gather is over; every error partial posted
    if (s == 0 && threadIdx.x == 0) {
      float t = 0.f;
      for (int r = 0; r < S; ++r) t += *cluster_map(&xch[1], (unsigned)r);  // rank order
      float* ep = q.err_part + (size_t)j * q.nb;
      ep[0] = t;
      for (int i = 1; i < q.nb; ++i) ep[i] = 0.f;
    }

    // ---- scatter the column slab back into the row slabs
    for (int e0 = threadIdx.x; e0 < nfar; e0 += 4 * blockDim.x) {
      float2 v[4];
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int e = e0 + q4 * blockDim.x;
        if (e < nfar) {
          const int k = e / (W * H), rem = e - k * (W * H), u = rem / H, cl = rem - u * H;
          v[q4] = CA[(k * H + cl) * PITCH + u];
        }
      }
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int e = e0 + q4 * blockDim.x;
        if (e < nfar) {
          const int k = e / (W * H), rem = e - k * (W * H), u = rem / H, cl = rem - u * H;
          const int ow = u / H;
          cluster_map(RA, (unsigned)ow)[(k * H + u - ow * H) * PITCH + r0 + cl] = v[q4];
        }
      }
    }
    cluster_sync();  // B3: every row slab holds its inverse-column-transformed rows

    // ---- inverse row DFTs: psi'_k (unnormalised by W^2, which the constraint
    // factor carries)
    for (int t0 = 0; t0 < M * H; t0 += NL) {
      const int t = t0 + line;
      const bool on = act && t < M * H;
      float2* row = RA + t * PITCH;  // row line t = k * H + r
      if (on && lane < G::N1) {
        float2 z[G::N2];
#pragma unroll
        for (int k2 = 0; k2 < G::N2; ++k2) z[k2] = row[lane + G::N1 * k2];
        inv_stepA<W>(z, lane, tw, lbuf);
      }
      line_sync<W>();
      if (on && lane < G::N2) {
        float2 v[G::N1];
        inv_stepB<W>(v, lane, lbuf);
#pragma unroll
        for (int n1 = 0; n1 < G::N1; ++n1) row[G::N2 * n1 + lane] = v[n1];
      }
      line_sync<W>();
    }
    __syncthreads();

    // ---- object update (written in place: the group's boxes are disjoint)
    // and the probe sums of this cluster's slot, on the row slab
    {
      const bool acc = !first || q.accumulate;
      const float omb = 1.f - q.a.beta, omg = 1.f - q.a.gamma, bom = q.a.beta * om;
      const int slot = cid;
      for (int e = threadIdx.x; e < H * W; e += blockDim.x) {
        const int r = e / W, c = e - r * W, gr = r0 + r;
        const float2 o = obuf[e];
        float* pd = q.pden + ((size_t)slot * W + gr) * W + c;
        const float pd0 = acc ? *pd : 0.f;
        float2 sT = make_float2(0.f, 0.f);
        float pint = 0.f;
        for (int k = 0; k < M; ++k) {
          const float2 p = pbuf[(k * H + r) * W + c];
          const float2 v = RA[(k * H + r) * PITCH + c];
          float2* pn = q.pnum + (((size_t)slot * M + k) * W + gr) * W + c;
          const float2 D = csub(v, cmul(p, o));
          sT = cadd(sT, cmulc(D, p));
          pint += cabs2(p);
          const float2 nm = cmulc(D, o);
          *pn = acc ? cadd(*pn, nm) : nm;
        }
        const float dn = fmaf(omg, pint, gden);
        const float sc = dn > 0.f ? q.a.alpha_O / dn : 0.f;  // a zero denominator has a zero numerator
        const float2 onw = make_float2(fmaf(sc, sT.x, o.x), fmaf(sc, sT.y, o.y));
        q.O[(size_t)(cc.x + gr) * q.Hx + cc.y + c] = onw;
        if (q.refine == 1) obuf[e] = onw;
        const float dv = fmaf(omb, cabs2(o), bom);
        *pd = acc ? pd0 + dv : dv;
      }
      osum_local += om;
    }

    // ---- XCORR_A: forward row DFTs of the refined crop rows (registration
    // plane M + 1)
    if (q.refine == 1) {
      __syncthreads();
      for (int t0 = 0; t0 < H; t0 += NL) {
        const int t = t0 + line;
        const bool on = act && t < H;
        if (on && lane < G::N2) {
          float2 v[G::N1];
#pragma unroll
          for (int n1 = 0; n1 < G::N1; ++n1) v[n1] = obuf[t * W + G::N2 * n1 + lane];
          fwd_step1<W>(v, lane, tw, lbuf);
        }
        line_sync<W>();
        if (on && lane < G::N1) {
          float2 z[G::N2];
          fwd_step3<W>(z, lane, lbuf);
          float2* dst = q.scratch + (((size_t)lp * q.npl + M + 1) * W + r0 + t) * W;
#pragma unroll
          for (int k2 = 0; k2 < G::N2; ++k2) dst[lane + G::N1 * k2] = z[k2];
        }
        line_sync<W>();
      }
    }
    __syncthreads();  // obuf, lbuf and cbuf are refilled by the next patch
    first = false;
  }
  cluster_sync();  // no CTA leaves while another may still touch its shared memory
  if (s == 0 && threadIdx.x == 0 && !first)
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
  if (!f || M < 1 || S > 8) return g;
  int L = 16, LP = 0;
  switch (W) {
    case 32: patch_line<32>(L, LP); break;
    case 64: patch_line<64>(L, LP); break;
    case 96: patch_line<96>(L, LP); break;
    default: patch_line<128>(L, LP); break;
  }
  const int H = W / S;
  // lines per round: as many as the launch bound holds, at most one round
  g.NL = std::min(kPatchMaxThreads / L, M * H);
  g.NT = kPatchMaxThreads;  // the element-wise phases use every thread
  g.sm = (size_t)(W + 2 * M * H * (W + 1) + g.NL * LP + H * W + M * H * W) * sizeof(float2) +
         (size_t)W * H * sizeof(uint16_t);
  if (g.sm > (size_t)smem_optin() - 512) return g;
  if (allow_max_smem(f) != cudaSuccess) {
    cudaGetLastError();
    return g;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S);
  cfg.blockDim = dim3(g.NT);
  cfg.dynamicSmemBytes = g.sm;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = S;
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
  cfg.gridDim = dim3(nclusters * g.S);
  cfg.blockDim = dim3(g.NT);
  cfg.dynamicSmemBytes = g.sm;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g.S;
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
