// Host side of libpty: the C ABI declared in include/pty.h.
//
// The handle owns every device array of one reconstruction problem.  One
// M-rPIE iteration (M-rPIE section of Guzzi et al., arXiv 2205.04295) is run
// as: round the positions to crop corners, partition them into groups of
// pairwise-disjoint boxes (greedy first fit), and for each group, for each
// chunk of at most Qc patches, launch the three passes (rows_fwd, cols,
// rows_inv), then apply the group's probe update.  Qc is set so that the
// chunk's far-field waves (Qc * M * W^2 complex64) fit the scratch budget and
// stay resident in L2.
#include "pty_internal.h"
#include "../../include/pty.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return fail(PTY_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                        \
  } while (0)

#define TRY(call)              \
  do {                         \
    int r_ = (call);           \
    if (r_ != PTY_OK) return r_; \
  } while (0)

__global__ void k_sum_u16(const uint16_t* __restrict__ I, size_t n,
                          unsigned long long* out) {
  unsigned long long s = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    s += I[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);  // integer: exact in any order
}

// Copy patterns ids[0..n) (W2 counts each, W2 a multiple of 8) from host
// memory the device can address (page-locked, unified addressing) into the
// device stack, and add their counts to *sum (integers: exact in any order).
// Reads cross the host link; one launch moves a whole group.  It runs beside
// the passes, so it is kept small: 4 CTAs, each thread with 8 independent
// 16-byte reads in flight (128 KB, enough to cover the link's latency at its
// bandwidth); 64 CTAs with one read each took SM slots from the passes
// (62.5 -> 59.3 ms for an end-to-end iteration of the 10^4-pattern spiral).
constexpr int kGatherCtas = 4;
__global__ void k_gather_host(uint16_t* __restrict__ dst, const uint16_t* __restrict__ src,
                              const int* __restrict__ ids, int n, int W2,
                              unsigned long long* sum) {
  const int per = W2 / 8;  // 16-byte vectors per pattern
  const long long total = (long long)n * per;
  unsigned long long s = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < total;
       i0 += 8 * stride) {
    uint4 v[8];
    size_t o[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = i0 + u * stride;
      if (i < total) {
        const int p = (int)(i / per), e = (int)(i - (long long)p * per);
        o[u] = (size_t)ids[p] * W2 + (size_t)e * 8;
        v[u] = *reinterpret_cast<const uint4*>(src + o[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (i0 + u * stride < total) {
        *reinterpret_cast<uint4*>(dst + o[u]) = v[u];
        const unsigned w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) s += (w[q] & 0xffffu) + (w[q] >> 16);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(sum, s);
}

__global__ void k_iota(int* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = i;
}

// Boxes with corners a, b overlap iff |a.y - b.y| < W and |a.x - b.x| < W;
// only the 3x3 neighbouring cells of a W-sized grid can hold such a corner.
int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// First-fit grouping in scan order into groups of pairwise-disjoint W x W
// boxes.  Exact tests use a per-group table over a W-sized grid (two corners
// in one W x W cell always overlap, so a group holds at most one member per
// cell: 3 x 3 lookups).  A finer grid (cells of W/4) keeps, per cell, a
// bitset of the groups whose clash zone (|dy| < W and |dx| < W around a
// member) covers the whole cell: those groups certainly clash, so a position
// exact-tests only the groups whose bit is clear, in order.  The result is
// the plain first fit.
void greedy_group(const std::vector<int2>& c, int W, const int32_t* order,
                  int max_group, std::vector<int>& gptr, std::vector<int>& gpos) {
  const int N = (int)c.size();
  int miny = 0, minx = 0, maxy = 0, maxx = 0;
  for (int j = 0; j < N; ++j) {
    if (j == 0 || c[j].x < miny) miny = c[j].x;
    if (j == 0 || c[j].y < minx) minx = c[j].y;
    if (j == 0 || c[j].x > maxy) maxy = c[j].x;
    if (j == 0 || c[j].y > maxx) maxx = c[j].y;
  }
  // W grid: one member per group and cell (exact tests)
  const int ncy = (maxy - miny) / W + 1, ncx = (maxx - minx) / W + 1;
  const size_t ncell = (size_t)ncy * ncx;
  // fine grid: per cell, the groups whose clash zone covers the whole cell
  const int s = std::max(1, W / 4);
  const int nfy = (maxy - miny) / s + 1, nfx = (maxx - minx) / s + 1;
  const size_t nfine = (size_t)nfy * nfx;
  int words = 2;
  std::vector<uint64_t> cover(nfine * words, 0);
  std::vector<int> table;  // [group][cell] -> member or -1
  std::vector<int> gsize;
  std::vector<std::vector<int>> members;
  for (int n = 0; n < N; ++n) {
    const int j = order ? order[n] : n;
    const int jy = c[j].x, jx = c[j].y;
    const int cy = (jy - miny) / W, cx = (jx - minx) / W;
    const size_t f = (size_t)((jy - miny) / s) * nfx + (jx - minx) / s;
    const int G = (int)members.size();
    int pick = G;
    const uint64_t* cv = cover.data() + f * words;
    for (int w = 0; w < words && pick == G; ++w) {
      uint64_t free_ = ~cv[w];
      while (free_) {
        const int g = w * 64 + __builtin_ctzll(free_);
        free_ &= free_ - 1;
        if (g >= G) break;
        if (max_group > 0 && gsize[g] >= max_group) continue;
        const int* tg = table.data() + (size_t)g * ncell;
        bool clash = false;
        for (int dy = -1; dy <= 1 && !clash; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int yy = cy + dy, xx = cx + dx;
            if (yy < 0 || xx < 0 || yy >= ncy || xx >= ncx) continue;
            const int i = tg[(size_t)yy * ncx + xx];
            if (i >= 0 && std::abs(c[i].x - jy) < W && std::abs(c[i].y - jx) < W) {
              clash = true;
              break;
            }
          }
        if (!clash) { pick = g; break; }
      }
    }
    if (pick == G) {
      if (G == words * 64) {
        std::vector<uint64_t> c2(nfine * words * 2, 0);
        for (size_t q = 0; q < nfine; ++q)
          std::copy(cover.begin() + q * words, cover.begin() + (q + 1) * words, c2.begin() + q * words * 2);
        cover.swap(c2);
        words *= 2;
      }
      members.emplace_back();
      gsize.push_back(0);
      table.resize(table.size() + ncell, -1);
    }
    const int g = pick;
    members[g].push_back(j);
    ++gsize[g];
    table[(size_t)g * ncell + (size_t)cy * ncx + cx] = j;
    // fine cells wholly inside j's clash zone (iy - W, iy + W) x (ix - W, ix + W)
    const int fy0 = std::max(0, -floordiv(-(jy - W + 1 - miny), s));
    const int fy1 = std::min(nfy - 1, floordiv(jy + W - s - miny, s));
    const int fx0 = std::max(0, -floordiv(-(jx - W + 1 - minx), s));
    const int fx1 = std::min(nfx - 1, floordiv(jx + W - s - minx, s));
    const uint64_t bit = 1ull << (g & 63);
    for (int fy = fy0; fy <= fy1; ++fy)
      for (int fx = fx0; fx <= fx1; ++fx) cover[((size_t)fy * nfx + fx) * words + (g >> 6)] |= bit;
  }
  gptr.assign(members.size() + 1, 0);
  gpos.clear();
  gpos.reserve(N);
  for (size_t g = 0; g < members.size(); ++g) {
    gpos.insert(gpos.end(), members[g].begin(), members[g].end());
    gptr[g + 1] = (int)gpos.size();
  }
}

bool valid_perm(const int32_t* order, int N) {
  std::vector<char> seen(N, 0);
  for (int i = 0; i < N; ++i) {
    if (order[i] < 0 || order[i] >= N || seen[order[i]]) return false;
    seen[order[i]] = 1;
  }
  return true;
}

}  // namespace

int pty::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

struct pty_handle {
  int W = 0, M = 0, N = 0, Hy = 0, Hx = 0;
  cudaStream_t stream = nullptr;
  pty_alloc_fn af = nullptr;
  pty_free_fn ff = nullptr;
  void* actx = nullptr;
  int device = 0;
  int flags = 0;             // PTY_FLAG_* of the problem description
  pty::Tiling tl{}, tlr{};   // plain and refining launch geometry
  int Qc = 1, Qcr = 1, nslots = 1;
  pty::PatchGeo pg{};        // fused patch kernel (pg.S > 0: it replaces the three passes)
  pty::RefGeo rg{};
  float2* roots = nullptr;
  float2* upart = nullptr;  // fine-grid partial sums of the registration
  int* updone = nullptr;     // N counters of finished CTAs per patch (tensor-core form)
  int roots_U = 0;
  float *cval = nullptr, *gap = nullptr;
  int* cidx = nullptr;
  // differentiable form: its own grouping ((W+1)-boxes at floor corners)
  int Qcg = 1;
  std::vector<float> gpos_key;
  std::vector<int> ggptr, ggpos;
  int* ggpos_d = nullptr;
  float* gpos_part = nullptr;
  float inv_w = 1.f;
  // device state
  float2 *O = nullptr, *P = nullptr, *tw = nullptr, *scratch = nullptr, *pnum = nullptr;
  uint16_t* I = nullptr;
  float *pos = nullptr, *am = nullptr, *av = nullptr, *pden = nullptr, *osum = nullptr;
  float *omax_part = nullptr, *err_part = nullptr, *pmax_part = nullptr, *err_iter = nullptr;
  float* shift = nullptr;
  int2* corners = nullptr;
  int *gpos_d = nullptr, *iota = nullptr, *flag = nullptr;
  unsigned long long* sum_d = nullptr;
  size_t err_part_n = 0;
  int err_iter_cap = 0;
  // host state
  double sumI = 0.0;
  bool has_data = false;
  int adam_t = 0, iter = 0;
  std::vector<float> pos_h;
  std::vector<int2> corners_h;
  std::vector<int> gptr, gpos;
  std::vector<int32_t> order;
  bool groups_valid = false;
  int grouped_max = -1;
  std::vector<int2> grouped_corners;  // inputs of the current groups
  std::vector<int32_t> grouped_order;
  std::vector<void*> allocs;
  // accounting
  int prof_mode = 0;
  long long n_launch[PTY_K_COUNT] = {0};
  double ms[PTY_K_COUNT] = {0};
  long long patches = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> event_pool;
  // One captured plain iteration, replayed while nothing its launch
  // arguments depend on has changed.  `epoch` counts such changes (groups
  // rebuilt, tiling or buffers replaced, new data).
  unsigned long long epoch = 0, iter_epoch = ~0ull;
  cudaGraphExec_t iter_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  pty_rpie_params iter_params{};
  long long iter_launch[PTY_K_COUNT] = {0};
  long long iter_patches = 0;
  // tensor maps of the scratch for the column pass's TMA staging (plain and
  // registration tilings); tma_err[0] is set by a wait of a staged pass that
  // timed out, tma_err[1] is the stalled-copy test hook (pty_debug_stall_copies)
  CUtensorMap tmap_b{}, tmap_br{};
  bool tma_b = false, tma_br = false;
  int* tma_err = nullptr;
  size_t scratch_n = 0;  // complex elements allocated in the scratch
  double* modes_G = nullptr;  // Gram matrix of the probe modes (M*M complex double)
  float2* modes_V = nullptr;  // their eigenvectors, as the mixing matrix
  float* err_slot = nullptr;  // the captured iteration's error
  double* err_dpart = nullptr;  // the error reduction's per-CTA partial sums
  bool graphs_off = false;    // capture failed once: launch directly
  // A host pattern stack whose upload pty_set_data_async deferred: the next
  // pty_run_iterations copies it group by group on up_stream (one event per
  // group) while the compute stream runs earlier groups.
  const uint16_t* up_host = nullptr;
  const uint16_t* up_dev = nullptr;  // up_host as the device addresses it, if it can
  int up_next = 0;
  cudaStream_t up_stream = nullptr;
  std::vector<cudaEvent_t> up_ev;
  cudaEvent_t up_done = nullptr;
  bool sum_host_valid = false;  // sumI matches sum_d

  cudaEvent_t take_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // Launch-accounting bracket around one kernel launch of kind k.
  struct Mark {
    pty_handle* h;
    int k;
    cudaEvent_t a = nullptr;
    Mark(pty_handle* hh, int kk) : h(hh), k(kk) {
      ++h->n_launch[k];
      if (h->prof_mode) {
        a = h->take_event();
        cudaEventRecord(a, h->stream);
      }
    }
    ~Mark() {
      if (a) {
        cudaEvent_t b = h->take_event();
        cudaEventRecord(b, h->stream);
        h->pending.push_back({k, {a, b}});
      }
    }
  };
  void drain() {
    for (auto& p : pending) {
      float t = 0.f;
      cudaEventSynchronize(p.second.second);
      cudaEventElapsedTime(&t, p.second.first, p.second.second);
      ms[p.first] += t;
      event_pool.push_back(p.second.first);
      event_pool.push_back(p.second.second);
    }
    pending.clear();
  }

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (af) {
      p = af(bytes, stream, actx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) allocs.push_back(p);
    return p;
  }
  void dfree(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) allocs.erase(it);
    if (ff) ff(p, stream, actx);
    else cudaFree(p);
  }
  ~pty_handle() {
    if (stream) cudaStreamSynchronize(stream);
    else cudaDeviceSynchronize();
    drain();
    if (iter_exec) cudaGraphExecDestroy(iter_exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (up_stream) cudaStreamSynchronize(up_stream);
    for (cudaEvent_t e : up_ev) cudaEventDestroy(e);
    if (up_done) cudaEventDestroy(up_done);
    if (up_stream) cudaStreamDestroy(up_stream);
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    for (void* p : allocs) {
      if (ff) ff(p, stream, actx);
      else cudaFree(p);
    }
  }
};

namespace {

template <class T>
int alloc_into(pty_handle* h, T*& p, size_t count) {
  p = static_cast<T*>(h->dalloc(count * sizeof(T)));
  if (!p) return fail(PTY_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
  return PTY_OK;
}

cudaMemcpyKind kind_in(int mem_kind) {
  return mem_kind == PTY_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
}
cudaMemcpyKind kind_out(int mem_kind) {
  return mem_kind == PTY_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}

int check_mem_kind(int mk) {
  if (mk != PTY_MEM_HOST && mk != PTY_MEM_DEVICE) return fail(PTY_EINVAL, "bad mem_kind %d", mk);
  return PTY_OK;
}

int check_params(const pty_rpie_params* p) {
  if (!p) return fail(PTY_EINVAL, "null rpie params");
  const float v[6] = {p->alpha_O, p->alpha_P, p->beta, p->gamma, p->eps, p->reg_eps};
  for (float x : v)
    if (!std::isfinite(x)) return fail(PTY_EINVAL, "non-finite rpie parameter");
  if (p->max_group < 0) return fail(PTY_EINVAL, "max_group < 0");
  if (p->eps < 0.f) return fail(PTY_EINVAL, "eps < 0");
  return PTY_OK;
}

// Round host positions, check the boxes, rebuild groups if needed.
int regroup(pty_handle* h, int max_group) {
  if (h->groups_valid && h->grouped_max == max_group) return PTY_OK;
  const int N = h->N, W = h->W;
  h->corners_h.resize(N);
  for (int j = 0; j < N; ++j) {
    const double y = h->pos_h[2 * j], x = h->pos_h[2 * j + 1];
    if (!std::isfinite(y) || !std::isfinite(x))
      return fail(PTY_EDATA, "position %d is not finite", j);
    const int cy = (int)std::floor(y + 0.5), cx = (int)std::floor(x + 0.5);
    if (cy < 0 || cx < 0 || cy + W > h->Hy || cx + W > h->Hx)
      return fail(PTY_EDATA, "crop box of position %d (corner %d,%d) leaves the %dx%d object",
                  j, cy, cx, h->Hy, h->Hx);
    h->corners_h[j] = make_int2(cy, cx);
  }
  // the grouping is a function of the corners, the scan order and max_group
  // only: unchanged inputs (same scan with new data, registration steps that
  // move no corner) keep the groups already on the device
  if (h->grouped_max == max_group && !h->gptr.empty() && h->grouped_order == h->order &&
      h->grouped_corners.size() == (size_t)N &&
      std::memcmp(h->grouped_corners.data(), h->corners_h.data(), sizeof(int2) * N) == 0) {
    h->groups_valid = true;
    return PTY_OK;
  }
  greedy_group(h->corners_h, W, h->order.empty() ? nullptr : h->order.data(), max_group,
               h->gptr, h->gpos);
  h->grouped_corners = h->corners_h;
  h->grouped_order = h->order;
  CU(cudaMemcpyAsync(h->corners, h->corners_h.data(), sizeof(int2) * N,
                     cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(h->gpos_d, h->gpos.data(), sizeof(int) * N, cudaMemcpyHostToDevice,
                     h->stream));
  h->groups_valid = true;
  h->grouped_max = max_group;
  ++h->epoch;
  return PTY_OK;
}

pty::UpdArgs upd_args(const pty_rpie_params* p) {
  return pty::UpdArgs{p->alpha_O, p->alpha_P, p->beta, p->gamma, p->eps, p->reg_eps};
}

// Registration (mode 1 XCORR_A, 2 XCORR_B) of patches [b0, b0 + nb) of the
// current grouping, whose crop planes the passes left in scratch patch slots
// 0 .. nb - 1 (planes M, M + 1 of the registration tiling).
int run_registration(pty_handle* h, int b0, int nb, int mode) {
  if (nb <= 0 || mode == 0) return PTY_OK;
  const int* ids = h->gpos_d + b0;
  const int npl = h->tlr.npl;
  pty_handle::Mark m(h, PTY_K_REFINE);
  if (mode == 2 || h->pg.S == 0) {
    // XCORR_B: both detector-plane images; XCORR_A on the three passes: the
    // refined crop, which pass C stores untransformed
    CU(pty::launch_xcorrb_rows(h->rg, h->scratch, npl, mode == 2 ? h->M : h->M + 1,
                               mode == 2 ? 2 : 1, nb, h->tw, h->stream));
    h->n_launch[PTY_K_REFINE] += 1;
  }
  CU(pty::launch_xcorr_cols(h->rg, h->scratch, npl, h->M, nb, h->tw, h->stream));
  CU(pty::launch_xcorr_rows(h->rg, h->scratch, npl, h->M, nb, h->tw, h->cval, h->cidx,
                            h->stream));
  CU(pty::launch_updft(h->rg, h->scratch, npl, h->M, ids, nb, h->cval, h->cidx, h->roots,
                       h->upart, h->shift, h->gap, h->updone, h->tma_err, h->stream));
  h->n_launch[PTY_K_REFINE] += 2;
  return PTY_OK;
}

// refine: 0 = plain, 1 = XCORR_A, 2 = XCORR_B registration of every patch.
// boff >= 0 (refining): the group is one chunk whose planes sit in scratch
// patch slots boff .. boff + n - 1, and its registration is left to the
// caller (run_registration over a batch of consecutive groups); boff < 0:
// chunks of the scratch budget, each registered at once.
// One group on the fused patch kernel: without registration the whole group
// in one launch (no scratch), with it in chunks of the registration's scratch
// planes, each chunk followed by the registration kernels.
int run_group_fused(pty_handle* h, int g, const pty_rpie_params* p, int refine, int boff) {
  const int n = h->gptr[g + 1] - h->gptr[g];
  const int* ids = h->gpos_d + h->gptr[g];
  const pty::Tiling& tl = refine ? h->tlr : h->tl;
  const int Qc = refine ? h->Qcr : n;
  pty::PatchArgs a = {};
  a.O = h->O; a.Hx = h->Hx; a.M = h->M; a.P = h->P; a.I = h->I; a.corners = h->corners;
  a.tw = h->tw; a.inv_w = h->inv_w; a.a = upd_args(p);
  a.pmax_part = h->pmax_part; a.n_pmax = h->tl.n_pmax;
  a.pnum = h->pnum; a.pden = h->pden; a.osum = h->osum;
  a.err_part = h->err_part; a.nb = h->W / tl.CB;  // the stride the error reduction reads
  a.scratch = h->scratch + (boff > 0 ? (size_t)boff * tl.npl * h->W * h->W : 0);
  a.npl = tl.npl; a.refine = refine;
  int used = 0;
  for (int c0 = 0; c0 < n; c0 += Qc) {
    const int nc = std::min(Qc, n - c0);
    const int* idc = ids + c0;
    a.ids = idc;
    a.npatch = nc;
    a.accumulate = c0 > 0;
    const int ncl = std::min(h->pg.ncap, nc);
    used = std::max(used, ncl);
    {
      pty_handle::Mark m(h, PTY_K_PATCH);
      CU(pty::launch_patch(h->pg, a, ncl, h->stream));
    }
    if (refine && boff < 0) {
      pty_handle::Mark m(h, PTY_K_REFINE);
      if (refine == 2) {
        CU(pty::launch_xcorrb_rows(h->rg, h->scratch, tl.npl, h->M, 2, nc, h->tw, h->stream));
        h->n_launch[PTY_K_REFINE] += 1;
      }
      CU(pty::launch_xcorr_cols(h->rg, h->scratch, tl.npl, h->M, nc, h->tw, h->stream));
      CU(pty::launch_xcorr_rows(h->rg, h->scratch, tl.npl, h->M, nc, h->tw, h->cval, h->cidx,
                                h->stream));
      CU(pty::launch_updft(h->rg, h->scratch, tl.npl, h->M, idc, nc, h->cval, h->cidx,
                           h->roots, h->upart, h->shift, h->gap, h->updone, h->tma_err,
                           h->stream));
      h->n_launch[PTY_K_REFINE] += 2;
    }
  }
  if (p->update_probe) {
    pty_handle::Mark m(h, PTY_K_PROBE);
    CU(pty::launch_probe_apply(h->tl, h->P, h->pnum, h->pden, h->osum, used, p->alpha_P,
                               p->reg_eps, h->pmax_part, h->stream));
  }
  h->patches += n;
  return PTY_OK;
}

int run_group(pty_handle* h, int g, const pty_rpie_params* p, int refine = 0, int boff = -1) {
  if (h->pg.S > 0) return run_group_fused(h, g, p, refine, boff);
  const int n = h->gptr[g + 1] - h->gptr[g];
  const int* ids = h->gpos_d + h->gptr[g];
  const pty::UpdArgs a = upd_args(p);
  const pty::Tiling& tl = refine ? h->tlr : h->tl;
  const int Qc = refine ? h->Qcr : h->Qc;
  // the batch slot of the group's first patch (its planes in the scratch)
  const int p0 = boff > 0 ? boff : 0;
  float2* scr = h->scratch + (size_t)p0 * tl.npl * h->W * h->W;
  // passes A and B take patches per CTA re-chosen for the chunk's size
  for (int c0 = 0; c0 < n; c0 += Qc) {
    const int nc = std::min(Qc, n - c0);
    const int* idc = ids + c0;
    const pty::Tiling tc = pty::tiling_for_chunk(tl, nc);
    {
      pty_handle::Mark m(h, PTY_K_ROWS_FWD);
      CU(pty::launch_rows_fwd(tc, h->O, h->Hx, h->P, idc, h->corners, nc, h->tw, scr,
                              h->omax_part, h->stream));
    }
    {
      pty_handle::Mark m(h, PTY_K_COLS);
      CU(pty::launch_cols(tc, scr, h->I, idc, nc, h->tw, h->inv_w, p->eps,
                          h->err_part,
                          refine ? (h->tma_br ? &h->tmap_br : nullptr) : (h->tma_b ? &h->tmap_b : nullptr),
                          h->tma_err, h->stream, refine == 2 ? h->M : -1, p0 * tl.npl));
    }
    {
      pty_handle::Mark m(h, PTY_K_ROWS_INV);
      CU(pty::launch_rows_inv(tc, h->O, h->Hx, h->P, idc, h->corners, nc, scr,
                              h->omax_part, h->pmax_part, h->tw, a, h->pnum, h->pden, h->osum,
                              c0 > 0, h->tma_err, h->stream, refine == 1 ? 1 : 0));
    }
    if (refine && boff < 0) {
      pty_handle::Mark m(h, PTY_K_REFINE);
      {
        // XCORR_B: both detector-plane images; XCORR_A: the refined crop,
        // which pass C stores untransformed
        CU(pty::launch_xcorrb_rows(h->rg, h->scratch, tl.npl, refine == 2 ? h->M : h->M + 1,
                                   refine == 2 ? 2 : 1, nc, h->tw, h->stream));
        h->n_launch[PTY_K_REFINE] += 1;
      }
      CU(pty::launch_xcorr_cols(h->rg, h->scratch, tl.npl, h->M, nc, h->tw, h->stream));
      CU(pty::launch_xcorr_rows(h->rg, h->scratch, tl.npl, h->M, nc, h->tw, h->cval, h->cidx,
                                h->stream));
      CU(pty::launch_updft(h->rg, h->scratch, tl.npl, h->M, idc, nc, h->cval, h->cidx,
                           h->roots, h->upart, h->shift, h->gap, h->updone, h->tma_err,
                           h->stream));
      h->n_launch[PTY_K_REFINE] += 2;
    }
  }
  if (p->update_probe) {
    const int used = (std::min(Qc, n) + tl.ppcc - 1) / tl.ppcc;
    pty_handle::Mark m(h, PTY_K_PROBE);
    CU(pty::launch_probe_apply(tl, h->P, h->pnum, h->pden, h->osum, used, p->alpha_P,
                               p->reg_eps, h->pmax_part, h->stream));
  }
  h->patches += n;
  return PTY_OK;
}

int ensure_err_cap(pty_handle* h, int n) {
  if (n <= h->err_iter_cap) return PTY_OK;
  if (h->err_iter) {
    CU(cudaStreamSynchronize(h->stream));
    h->dfree(h->err_iter);
  }
  h->err_iter = nullptr;
  h->err_iter_cap = 0;
  TRY(alloc_into(h, h->err_iter, (size_t)std::max(n, 64)));
  h->err_iter_cap = std::max(n, 64);
  return PTY_OK;
}

int finish_upload(pty_handle* h);

// (Re)encode the scratch's tensor maps for the current tilings; a tiling the
// TMA rules do not admit stages with cp.async instead.
void remap_scratch(pty_handle* h) {
  const size_t planes = h->scratch_n / ((size_t)h->W * h->W);
  h->tma_b = pty::encode_far_field_map(h->scratch, h->W, planes, h->tl.CB, &h->tmap_b);
  h->tma_br = pty::encode_far_field_map(h->scratch, h->W, planes, h->tlr.CB, &h->tmap_br);
}

// A wait of a staged pass (column pass TMA, inverse-row bulk copies) that
// timed out (reported at synchronising calls).
int check_tma_error(pty_handle* h) {
  int f = 0;
  CU(cudaMemcpyAsync(&f, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (f) {
    CU(cudaMemsetAsync(h->tma_err, 0, sizeof(int), h->stream));
    return fail(PTY_ETIMEOUT, "a staged copy (column or inverse-row pass) did not complete in time");
  }
  return PTY_OK;
}

// need_data: the call reads the data, so a deferred upload is completed first.
int check_handle(pty_handle* h, bool need_data) {
  if (!h) return fail(PTY_EINVAL, "null handle");
  if (need_data && !h->has_data) return fail(PTY_ESTATE, "pty_set_data has not been called");
  CU(cudaSetDevice(h->device));
  if (need_data && h->up_host) TRY(finish_upload(h));
  return PTY_OK;
}

int finite_check(pty_handle* h, const void* dev, size_t nfloat, const char* what) {
  CU(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  CU(pty::launch_finite_check(static_cast<const float*>(dev), nfloat, h->flag, h->stream));
  int f = 0;
  CU(cudaMemcpyAsync(&f, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (f) return fail(PTY_EDATA, "%s holds a non-finite value", what);
  return PTY_OK;
}

// Enqueue, on the upload stream, the copies of groups [up_next, g_end) of a
// pending host pattern stack (one cudaMemcpyAsync per run of consecutive
// pattern indices in the group) and record one event per group.
int upload_groups(pty_handle* h, int g_end) {
  const int G = (int)h->gptr.size() - 1;
  g_end = std::min(g_end, G);
  if (h->up_next >= g_end) return PTY_OK;
  const size_t W2 = (size_t)h->W * h->W;
  if (!h->up_stream) {
    // highest priority: its small gather kernels take SM slots ahead of the passes
    int lo = 0, hi = 0;
    CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CU(cudaStreamCreateWithPriority(&h->up_stream, cudaStreamNonBlocking, hi));
  }
  while ((int)h->up_ev.size() < G) {
    cudaEvent_t e = nullptr;
    CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->up_ev.push_back(e);
  }
  if (h->up_next == 0) {
    // the stack is overwritten only after everything already queued on the
    // compute stream (earlier iterations read it)
    CU(cudaEventRecord(h->up_ev[0], h->stream));
    CU(cudaStreamWaitEvent(h->up_stream, h->up_ev[0], 0));
    if (h->up_dev) CU(cudaMemsetAsync(h->sum_d, 0, sizeof(unsigned long long), h->up_stream));
  }
  for (; h->up_next < g_end; ++h->up_next) {
    const int g = h->up_next;
    if (h->up_dev) {
      // one gather kernel per group, summing the counts on the way
      k_gather_host<<<kGatherCtas, 256, 0, h->up_stream>>>(h->I, h->up_dev, h->gpos_d + h->gptr[g],
                                                   h->gptr[g + 1] - h->gptr[g], (int)W2,
                                                   h->sum_d);
      CU(cudaGetLastError());
      CU(cudaEventRecord(h->up_ev[g], h->up_stream));
      continue;
    }
    for (int i = h->gptr[g], b = h->gptr[g + 1]; i < b;) {
      const int j0 = h->gpos[i];
      int n = 1;
      while (i + n < b && h->gpos[i + n] == j0 + n) ++n;
      CU(cudaMemcpyAsync(h->I + (size_t)j0 * W2, h->up_host + (size_t)j0 * W2,
                         sizeof(uint16_t) * W2 * n, cudaMemcpyHostToDevice, h->up_stream));
      i += n;
    }
    CU(cudaEventRecord(h->up_ev[g], h->up_stream));
  }
  return PTY_OK;
}

// Complete a pending upload: the remaining groups, then the counts sum; the
// compute stream waits for both.
int finish_upload(pty_handle* h) {
  if (!h->up_host) return PTY_OK;
  TRY(upload_groups(h, (int)h->gptr.size() - 1));
  if (!h->up_dev) {  // the gather kernels summed the counts already
    const size_t W2 = (size_t)h->W * h->W;
    CU(cudaMemsetAsync(h->sum_d, 0, sizeof(unsigned long long), h->up_stream));
    k_sum_u16<<<296, 256, 0, h->up_stream>>>(h->I, (size_t)h->N * W2, h->sum_d);
    CU(cudaGetLastError());
  }
  if (!h->up_done) CU(cudaEventCreateWithFlags(&h->up_done, cudaEventDisableTiming));
  CU(cudaEventRecord(h->up_done, h->up_stream));
  CU(cudaStreamWaitEvent(h->stream, h->up_done, 0));
  h->up_host = nullptr;
  return PTY_OK;
}

// The host copy of sum(I), fetched once after a deferred or device upload.
int host_sum(pty_handle* h) {
  TRY(finish_upload(h));
  if (h->sum_host_valid) return PTY_OK;
  unsigned long long s = 0;
  CU(cudaMemcpyAsync(&s, h->sum_d, sizeof s, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->sumI = (double)s;
  h->sum_host_valid = true;
  return PTY_OK;
}

// pty_set_data and pty_set_data_async.  With defer and host memory the
// pattern stack is left pending: the next pty_run_iterations uploads it
// group by group (any other call that needs it uploads it whole first).
int set_data_impl(pty_handle* h, const uint16_t* I, const float* pos, const void* O0,
                  const void* P0, int mem_kind, bool defer) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (!I || !pos || !O0 || !P0) return fail(PTY_EINVAL, "null data pointer");
  const size_t W2 = (size_t)h->W * h->W;
  h->has_data = false;
  h->up_host = nullptr;  // a pending upload is superseded
  h->pos_h.resize(2 * (size_t)h->N);
  CU(cudaMemcpyAsync(h->pos_h.data(), pos, sizeof(float) * 2 * h->N,
                     mem_kind == PTY_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->groups_valid = false;
  TRY(regroup(h, 0));
  CU(cudaMemcpyAsync(h->pos, h->pos_h.data(), sizeof(float) * 2 * h->N, cudaMemcpyHostToDevice,
                     h->stream));
  CU(cudaMemcpyAsync(h->O, O0, sizeof(float2) * h->Hy * h->Hx, kind_in(mem_kind), h->stream));
  CU(cudaMemcpyAsync(h->P, P0, sizeof(float2) * h->M * W2, kind_in(mem_kind), h->stream));
  TRY(finite_check(h, h->O, (size_t)2 * h->Hy * h->Hx, "object"));
  TRY(finite_check(h, h->P, (size_t)2 * h->M * W2, "probe"));
  CU(cudaMemsetAsync(h->am, 0, sizeof(float) * 2 * h->N, h->stream));
  CU(cudaMemsetAsync(h->av, 0, sizeof(float) * 2 * h->N, h->stream));
  CU(cudaMemsetAsync(h->shift, 0, sizeof(float) * 2 * h->N, h->stream));
  CU(pty::launch_pmax(h->tl, h->P, h->pmax_part, h->stream));
  h->sum_host_valid = false;
  if (defer && mem_kind == PTY_MEM_HOST) {
    h->up_host = I;
    h->up_dev = nullptr;
    h->up_next = 0;
    // page-locked host memory the device can address is gathered by kernels;
    // anything else goes through cudaMemcpyAsync
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, I) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer && reinterpret_cast<uintptr_t>(pa.devicePointer) % 16 == 0 &&
        W2 % 8 == 0)
      h->up_dev = static_cast<const uint16_t*>(pa.devicePointer);
    cudaGetLastError();
  } else {
    CU(cudaMemcpyAsync(h->I, I, sizeof(uint16_t) * h->N * W2, kind_in(mem_kind), h->stream));
    CU(cudaMemsetAsync(h->sum_d, 0, sizeof(unsigned long long), h->stream));
    k_sum_u16<<<296, 256, 0, h->stream>>>(h->I, (size_t)h->N * W2, h->sum_d);
    CU(cudaGetLastError());
    if (!defer) TRY(host_sum(h));  // synchronises: the caller may reuse its buffers
  }
  h->adam_t = 0;
  h->iter = 0;
  h->has_data = true;
  ++h->epoch;
  return PTY_OK;
}

}  // namespace

extern "C" {

const char* pty_last_error(void) { return g_err.c_str(); }
int pty_abi_version(void) { return PTY_ABI_VERSION; }

int pty_init_problem(const pty_problem_desc* d, pty_handle** out) {
  g_err.clear();
  if (!d || !out) return fail(PTY_EINVAL, "null argument");
  *out = nullptr;
  if (!pty::supported_W(d->W)) return fail(PTY_EINVAL, "unsupported pattern size W=%d", d->W);
  if (d->M < 1 || d->M > 16) return fail(PTY_EINVAL, "M=%d outside 1..16", d->M);
  if (d->N < 1) return fail(PTY_EINVAL, "N=%d < 1", d->N);
  if (d->Hy < d->W || d->Hx < d->W) return fail(PTY_EINVAL, "object %dx%d smaller than W", d->Hy, d->Hx);
  if ((d->alloc == nullptr) != (d->free == nullptr))
    return fail(PTY_EINVAL, "alloc and free must be given together");
  if (d->flags & ~PTY_FLAG_FP32_REGISTRATION) return fail(PTY_EINVAL, "unknown flags 0x%x", d->flags);
  pty_handle* h = new (std::nothrow) pty_handle();
  if (!h) return fail(PTY_ENOMEM, "host allocation failed");
  h->W = d->W; h->M = d->M; h->N = d->N; h->Hy = d->Hy; h->Hx = d->Hx;
  h->stream = static_cast<cudaStream_t>(d->stream);
  h->af = d->alloc; h->ff = d->free; h->actx = d->alloc_ctx;
  h->flags = d->flags;
  auto bail = [&](int rc) { delete h; return rc; };
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(PTY_ECUDA, "no CUDA device"));
  }
  h->tl = pty::make_tiling(h->W, h->M, false);
  h->tlr = pty::make_tiling(h->W, h->M, true);
  if (cudaError_t e = pty::set_smem_limits(h->tl); e != cudaSuccess)
    return bail(fail(PTY_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)));
  pty::fill_residency(h->tl);
  pty::fill_residency(h->tlr);
  if (cudaError_t e = pty::set_grad_smem(h->tl); e != cudaSuccess)
    return bail(fail(PTY_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)));
  if (!pty::tiling_fits(h->tl) || !pty::tiling_fits(h->tlr))
    return bail(fail(PTY_EINVAL,
                     "W=%d with M=%d modes exceeds the per-CTA thread or shared-memory limits",
                     h->W, h->M));
  const size_t W2 = (size_t)h->W * h->W;
  const size_t budget = d->scratch_bytes ? d->scratch_bytes : ((size_t)64 << 20);
  h->Qc = (int)std::max<size_t>(1, budget / (W2 * h->tl.npl * sizeof(float2)));
  h->Qc = std::min(h->Qc, h->N);
  h->Qcr = (int)std::max<size_t>(1, budget / (W2 * h->tlr.npl * sizeof(float2)));
  h->Qcr = std::min(h->Qcr, h->N);
  h->Qcg = (int)std::max<size_t>(1, budget / (W2 * (h->M + 1) * sizeof(float2)));
  h->Qcg = std::min(h->Qcg, h->N);
  h->nslots = (std::max(std::max(h->Qc, h->Qcr), h->Qcg) + h->tl.ppc - 1) / h->tl.ppc;
  h->inv_w = (float)(1.0 / h->W);
  const int nrb = h->W / std::min(h->tl.R, h->tlr.R);
  const size_t scratch_elems =
      std::max(std::max((size_t)h->Qc * h->tl.npl, (size_t)h->Qcr * h->tlr.npl),
               (size_t)h->Qcg * (h->M + 1)) * W2;
  const size_t nparts = (size_t)h->Qcr * h->W;  // >= Qcr * (W / RX)
  h->err_part_n = (size_t)h->N * (h->W / h->tl.CB);
  const size_t err_part_cap = (size_t)h->N * (h->W / 2);  // any column block >= 2
  int rc = PTY_OK;
  if ((rc = alloc_into(h, h->O, (size_t)h->Hy * h->Hx)) ||
      (rc = alloc_into(h, h->P, (size_t)h->M * W2)) ||
      (rc = alloc_into(h, h->tw, (size_t)h->W)) ||
      (rc = alloc_into(h, h->scratch, scratch_elems)) ||
      (rc = alloc_into(h, h->tma_err, (size_t)2)) ||
      (rc = alloc_into(h, h->err_dpart, (size_t)pty::kErrPartsMax)) ||
      (rc = alloc_into(h, h->cval, nparts)) ||
      (rc = alloc_into(h, h->cidx, nparts)) ||
      (rc = alloc_into(h, h->gap, (size_t)h->N)) ||
      (rc = alloc_into(h, h->updone, (size_t)h->N)) ||
      (rc = alloc_into(h, h->pnum, (size_t)h->nslots * h->M * W2)) ||
      (rc = alloc_into(h, h->pden, (size_t)h->nslots * W2)) ||
      (rc = alloc_into(h, h->osum, (size_t)h->nslots)) ||
      (rc = alloc_into(h, h->omax_part, (size_t)std::max(h->Qc, h->Qcr) * nrb)) ||
      (rc = alloc_into(h, h->err_part, err_part_cap)) ||
      (rc = alloc_into(h, h->pmax_part, (size_t)h->tl.n_pmax)) ||
      (rc = alloc_into(h, h->I, (size_t)h->N * W2)) ||
      (rc = alloc_into(h, h->pos, (size_t)2 * h->N)) ||
      (rc = alloc_into(h, h->am, (size_t)2 * h->N)) ||
      (rc = alloc_into(h, h->av, (size_t)2 * h->N)) ||
      (rc = alloc_into(h, h->shift, (size_t)2 * h->N)) ||
      (rc = alloc_into(h, h->corners, (size_t)h->N)) ||
      (rc = alloc_into(h, h->gpos_d, (size_t)h->N)) ||
      (rc = alloc_into(h, h->ggpos_d, (size_t)h->N)) ||
      // dL/dpos partials: one pair per position and row block; sized for any
      // row-block height R >= 1 so that pty_set_tiling never outgrows it
      (rc = alloc_into(h, h->gpos_part, (size_t)h->N * h->W * 2)) ||
      (rc = alloc_into(h, h->iota, (size_t)h->N)) ||
      (rc = alloc_into(h, h->flag, (size_t)4)) ||
      (rc = alloc_into(h, h->sum_d, (size_t)1)))
    return bail(rc);
  h->scratch_n = scratch_elems;
  remap_scratch(h);
  std::vector<float2> tw(h->W);
  pty::make_twiddles(h->W, tw.data());
  if (cudaMemcpyAsync(h->tw, tw.data(), sizeof(float2) * h->W, cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->err_part, 0, sizeof(float) * err_part_cap, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->tma_err, 0, 2 * sizeof(int), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(PTY_ECUDA, "initial copies failed"));
  }
  k_iota<<<64, 256, 0, h->stream>>>(h->iota, h->N);
  if (cudaGetLastError() != cudaSuccess) return bail(fail(PTY_ECUDA, "iota launch failed"));
  *out = h;
  return PTY_OK;
}

int pty_destroy(pty_handle* h) {
  if (!h) return PTY_OK;
  cudaSetDevice(h->device);
  delete h;
  return PTY_OK;
}

int pty_set_data(pty_handle* h, const uint16_t* I, const float* pos, const void* O0,
                 const void* P0, int mem_kind) {
  return set_data_impl(h, I, pos, O0, P0, mem_kind, false);
}

int pty_set_data_async(pty_handle* h, const uint16_t* I, const float* pos, const void* O0,
                       const void* P0, int mem_kind) {
  return set_data_impl(h, I, pos, O0, P0, mem_kind, true);
}

int pty_set_scan_order(pty_handle* h, const int32_t* order) {
  g_err.clear();
  if (!h) return fail(PTY_EINVAL, "null handle");
  if (!order) {
    h->order.clear();
  } else {
    if (!valid_perm(order, h->N)) return fail(PTY_EINVAL, "scan order is not a permutation of 0..N-1");
    h->order.assign(order, order + h->N);
  }
  h->groups_valid = false;
  return PTY_OK;
}

// Capture one plain iteration (every group's passes and probe update, then
// the error reduction into err_slot) as a CUDA graph, unless the current one
// is still valid.  Captured on a private non-blocking stream (the caller's
// stream may be the legacy default stream, which cannot be captured) and
// launched on the caller's stream.  If capture or instantiation fails the
// handle falls back to direct launches of the same kernels.
int iteration_graph(pty_handle* h, const pty_rpie_params* p) {
  if (h->iter_exec && h->iter_epoch == h->epoch &&
      std::memcmp(&h->iter_params, p, sizeof *p) == 0)
    return PTY_OK;
  if (h->iter_exec) {
    CU(cudaGraphExecDestroy(h->iter_exec));
    h->iter_exec = nullptr;
  }
  if (!h->cap_stream) CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (!h->err_slot) TRY(alloc_into(h, h->err_slot, 1));
  long long l0[PTY_K_COUNT];
  std::memcpy(l0, h->n_launch, sizeof l0);
  const long long p0 = h->patches;
  cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  cudaGraph_t graph = nullptr;
  int rc = PTY_OK;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const int G = (int)h->gptr.size() - 1;
    for (int g = 0; g < G && rc == PTY_OK; ++g) rc = run_group(h, g, p);
    if (rc == PTY_OK) {
      pty_handle::Mark m(h, PTY_K_REDUCE);
      e = pty::launch_err_reduce(h->err_part, h->err_part_n, 0.0, h->sum_d, h->err_slot,
                                 h->err_dpart, h->stream);
    }
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e == cudaSuccess) e = e2;
  }
  h->stream = user;
  // the capture counted one iteration's launches: keep them per replay
  for (int k = 0; k < PTY_K_COUNT; ++k) {
    h->iter_launch[k] = h->n_launch[k] - l0[k];
    h->n_launch[k] = l0[k];
  }
  h->iter_patches = h->patches - p0;
  h->patches = p0;
  if (e == cudaSuccess && rc == PTY_OK) e = cudaGraphInstantiate(&h->iter_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != PTY_OK || e != cudaSuccess) {
    cudaGetLastError();
    h->iter_exec = nullptr;
    h->graphs_off = true;  // direct launches from now on
    g_err.clear();
    return PTY_OK;
  }
  h->iter_epoch = h->epoch;
  h->iter_params = *p;
  return PTY_OK;
}

int pty_run_iterations(pty_handle* h, int n_iter, const pty_rpie_params* p, float* err_out) {
  g_err.clear();
  TRY(check_handle(h, false));
  if (!h->has_data) return fail(PTY_ESTATE, "pty_set_data has not been called");
  TRY(check_params(p));
  if (n_iter < 0) return fail(PTY_EINVAL, "n_iter < 0");
  if (n_iter == 0) return finish_upload(h);
  TRY(ensure_err_cap(h, n_iter));
  for (int it = 0; it < n_iter; ++it) {
    TRY(regroup(h, p->max_group));
    if (h->up_host) {
      // first iteration after pty_set_data_async: group g waits only for its
      // own patterns, which were queued two groups ahead
      const int G = (int)h->gptr.size() - 1;
      for (int g = 0; g < G; ++g) {
        TRY(upload_groups(h, g + 3));
        CU(cudaStreamWaitEvent(h->stream, h->up_ev[g], 0));
        TRY(run_group(h, g, p));
      }
      TRY(finish_upload(h));  // the counts sum for the error
      {
        pty_handle::Mark m(h, PTY_K_REDUCE);
        CU(pty::launch_err_reduce(h->err_part, h->err_part_n, 0.0, h->sum_d, h->err_iter + it,
                                  h->err_dpart, h->stream));
      }
      ++h->iter;
      continue;
    }
    if (!h->prof_mode && !h->graphs_off) {
      TRY(iteration_graph(h, p));
      if (h->iter_exec) {
        CU(cudaGraphLaunch(h->iter_exec, h->stream));
        CU(cudaMemcpyAsync(h->err_iter + it, h->err_slot, sizeof(float),
                           cudaMemcpyDeviceToDevice, h->stream));
        for (int k = 0; k < PTY_K_COUNT; ++k) h->n_launch[k] += h->iter_launch[k];
        h->patches += h->iter_patches;
        ++h->iter;
        continue;
      }
    }
    const int G = (int)h->gptr.size() - 1;
    for (int g = 0; g < G; ++g) TRY(run_group(h, g, p));
    {
      pty_handle::Mark m(h, PTY_K_REDUCE);
      CU(pty::launch_err_reduce(h->err_part, h->err_part_n, 0.0, h->sum_d, h->err_iter + it,
                                h->err_dpart, h->stream));
    }
    ++h->iter;
  }
  if (err_out) {
    CU(cudaMemcpyAsync(err_out, h->err_iter, sizeof(float) * n_iter, cudaMemcpyDeviceToHost,
                       h->stream));
    TRY(check_tma_error(h));
  }
  return PTY_OK;
}

int pty_refine_positions(pty_handle* h, int n_iter, const pty_rpie_params* p,
                         const pty_refine_params* r, float* err_out, float* shift_out) {
  g_err.clear();
  TRY(check_handle(h, true));
  TRY(check_params(p));
  if (!r) return fail(PTY_EINVAL, "null refine params");
  if (n_iter < 0) return fail(PTY_EINVAL, "n_iter < 0");
  if (r->upsample < 1 || r->upsample > 40) return fail(PTY_EINVAL, "upsample %d outside 1..40", r->upsample);
  if (!std::isfinite(r->lr) || !(r->b1 >= 0.f && r->b1 < 1.f) || !(r->b2 >= 0.f && r->b2 < 1.f) ||
      !(r->eps >= 0.f) || !(r->max_step >= 0.f) || r->start_iter < 0 ||
      (r->point != PTY_XCORR_A && r->point != PTY_XCORR_B))
    return fail(PTY_EINVAL, "bad refine parameters");
  if (r->upsample != h->roots_U) {
    h->rg = pty::make_refgeo(h->W, r->upsample, !(h->flags & PTY_FLAG_FP32_REGISTRATION));
    if (h->rg.smU > 227 * 1024) return fail(PTY_EINVAL, "upsample %d too large for W=%d", r->upsample, h->W);
    CU(pty::set_refine_smem(h->rg));
    CU(pty::set_smem_limits(h->tlr));
    if (h->roots) {
      CU(cudaStreamSynchronize(h->stream));
      h->dfree(h->roots);
      h->roots = nullptr;
    }
    std::vector<float2> roots((size_t)h->rg.U * h->W);
    pty::make_up_roots(h->W, h->rg.U, roots.data());
    TRY(alloc_into(h, h->roots, roots.size()));
    if (h->upart) h->dfree(h->upart);
    h->upart = nullptr;
    TRY(alloc_into(h, h->upart, (size_t)h->Qcr * (h->W / 16) * h->rg.K * h->rg.K));
    CU(cudaMemcpyAsync(h->roots, roots.data(), sizeof(float2) * roots.size(),
                       cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->roots_U = r->upsample;
  }
  if (n_iter == 0) return PTY_OK;
  // the fine-grid kernels' per-patch counters start at zero (each launch
  // leaves them there; this also clears them after a launch that gave up)
  CU(cudaMemsetAsync(h->updone, 0, sizeof(int) * h->N, h->stream));
  TRY(ensure_err_cap(h, n_iter));
  for (int it = 0; it < n_iter; ++it) {
    TRY(regroup(h, p->max_group));
    const bool on = h->iter >= r->start_iter;
    if (on) CU(pty::set_smem_limits(h->tlr));
    const int G = (int)h->gptr.size() - 1;
    const int mode = on ? (r->point == PTY_XCORR_B ? 2 : 1) : 0;
    // The registration of a group changes nothing the later groups read (the
    // positions move at the end of the iteration), so it runs once per batch
    // of consecutive groups: patches [b0, b0 + nb) of the grouping, their
    // crop planes in scratch patch slots 0 .. nb - 1.
    int b0 = 0, nb = 0;
    for (int g = 0; g < G; ++g) {
      const int n = h->gptr[g + 1] - h->gptr[g];
      if (mode == 0) {
        TRY(run_group(h, g, p, 0));
        continue;
      }
      if (nb + n > h->Qcr) {  // the batch is full
        TRY(run_registration(h, b0, nb, mode));
        b0 = h->gptr[g];
        nb = 0;
      }
      if (n > h->Qcr) {  // a group larger than the scratch: chunks, each registered at once
        TRY(run_group(h, g, p, mode));
        b0 = h->gptr[g + 1];
        continue;
      }
      TRY(run_group(h, g, p, mode, nb));
      nb += n;
    }
    TRY(run_registration(h, b0, nb, mode));
    {
      // the partial sums of this iteration follow its column-pass tiling
      const size_t nerr = (size_t)h->N * (h->W / (on ? h->tlr.CB : h->tl.CB));
      pty_handle::Mark m(h, PTY_K_REDUCE);
      CU(pty::launch_err_reduce(h->err_part, nerr, 0.0, h->sum_d, h->err_iter + it, h->err_dpart,
                                h->stream));
    }
    if (on) {
      ++h->adam_t;
      const double bc1 = 1.0 - std::pow((double)r->b1, h->adam_t);
      const double bc2 = 1.0 - std::pow((double)r->b2, h->adam_t);
      {
        pty_handle::Mark m(h, PTY_K_REFINE);
        CU(pty::launch_adam(h->pos, h->am, h->av, h->shift, h->N, r->lr, r->b1, r->b2, r->eps,
                            (float)bc1, (float)bc2, r->max_step, (float)(h->Hy - h->W),
                            (float)(h->Hx - h->W), h->stream));
      }
      CU(cudaMemcpyAsync(h->pos_h.data(), h->pos, sizeof(float) * 2 * h->N,
                         cudaMemcpyDeviceToHost, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      h->groups_valid = false;
    }
    ++h->iter;
  }
  if (err_out) {
    CU(cudaMemcpyAsync(err_out, h->err_iter, sizeof(float) * n_iter, cudaMemcpyDeviceToHost,
                       h->stream));
  }
  if (shift_out) {
    CU(cudaMemcpyAsync(shift_out, h->shift, sizeof(float) * 2 * h->N, cudaMemcpyDeviceToHost,
                       h->stream));
  }
  CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

namespace {
// Validate device positions for the bilinear crop and (re)group them into
// (W+1)-boxes at floor corners when they changed.
int grad_prepare(pty_handle* h, const float* pos) {
  const int N = h->N, W = h->W;
  std::vector<float> ph(2 * (size_t)N);
  CU(cudaMemcpyAsync(ph.data(), pos, sizeof(float) * 2 * N, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (ph == h->gpos_key && !h->ggptr.empty()) return PTY_OK;
  std::vector<int2> c(N);
  for (int j = 0; j < N; ++j) {
    const float y = ph[2 * j], x = ph[2 * j + 1];
    if (!std::isfinite(y) || !std::isfinite(x)) return fail(PTY_EDATA, "position %d is not finite", j);
    const int iy = (int)std::floor(y), ix = (int)std::floor(x);
    if (iy < 0 || ix < 0 || iy + W + 1 > h->Hy || ix + W + 1 > h->Hx)
      return fail(PTY_EDATA, "bilinear crop of position %d leaves the %dx%d object", j, h->Hy, h->Hx);
    c[j] = make_int2(iy, ix);
  }
  greedy_group(c, W + 1, nullptr, 0, h->ggptr, h->ggpos);
  CU(cudaMemcpyAsync(h->ggpos_d, h->ggpos.data(), sizeof(int) * N, cudaMemcpyHostToDevice,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->gpos_key = ph;
  return PTY_OK;
}

int grad_run(pty_handle* h, const void* Ov, const void* Pv, const float* pos, float delta,
             float* loss, void* gOv, void* gPv, float* gpos, bool adjoint) {
  TRY(check_handle(h, true));
  if (!Ov || !Pv || !pos || !loss) return fail(PTY_EINVAL, "null argument");
  if (adjoint && (!gOv || !gPv || !gpos)) return fail(PTY_EINVAL, "null gradient output");
  if (!std::isfinite(delta) || delta < 0.f) return fail(PTY_EINVAL, "delta must be finite and >= 0");
  TRY(grad_prepare(h, pos));
  const float2* O = static_cast<const float2*>(Ov);
  const float2* P = static_cast<const float2*>(Pv);
  float2* gO = static_cast<float2*>(gOv);
  const int npl = h->M + 1;
  const size_t W2 = (size_t)h->W * h->W;
  if (adjoint) {
    CU(cudaMemsetAsync(gO, 0, sizeof(float2) * h->Hy * h->Hx, h->stream));
    CU(cudaMemsetAsync(h->pnum, 0, sizeof(float2) * h->nslots * h->M * W2, h->stream));
  }
  CU(cudaMemsetAsync(h->err_part, 0, sizeof(float) * h->err_part_n, h->stream));
  // Nothing is updated during the evaluation, so the per-patch passes take
  // full chunks of the group-ordered position list regardless of where the
  // groups end; only the scatter into dL/dO follows the groups (one launch
  // per group part in the chunk: disjoint boxes, no atomics, a fixed order).
  const int G = (int)h->ggptr.size() - 1;
  const int N = h->ggptr[G];
  int g = 0;
  for (int c0 = 0; c0 < N; c0 += h->Qcg) {
    const int nc = std::min(h->Qcg, N - c0);
    const int* idc = h->ggpos_d + c0;
    pty_handle::Mark m(h, PTY_K_GRAD);
    CU(pty::launch_grad_rows_fwd(h->tl, O, h->Hx, P, idc, pos, nc, h->tw, h->scratch, npl,
                                 h->stream));
    CU(pty::launch_cols_grad(h->tl, h->scratch, h->I, idc, nc, h->tw, h->inv_w, delta,
                             h->err_part, npl, h->tma_b ? &h->tmap_b : nullptr, h->tma_err,
                             h->stream));
    h->n_launch[PTY_K_GRAD] += 1;
    if (adjoint) {
      CU(pty::launch_grad_rows_inv(h->tl, O, h->Hx, P, idc, pos, nc, h->scratch, npl, h->tw,
                                   h->pnum, 1, h->gpos_part, h->stream));
      h->n_launch[PTY_K_GRAD] += 1;
      for (; g < G && h->ggptr[g] < c0 + nc; ++g) {
        const int a = std::max(h->ggptr[g], c0), b = std::min(h->ggptr[g + 1], c0 + nc);
        CU(pty::launch_grad_scatter(h->W, h->M, gO, h->Hx, h->ggpos_d + a, pos, b - a,
                                    h->scratch + (size_t)(a - c0) * npl * W2, npl,
                                    h->stream));
        h->n_launch[PTY_K_GRAD] += 1;
        if (h->ggptr[g + 1] > c0 + nc) break;  // the group continues in the next chunk
      }
    }
  }
  const int used = (std::min(h->Qcg, h->N) + h->tl.ppc - 1) / h->tl.ppc;
  pty_handle::Mark m(h, PTY_K_GRAD);
  CU(pty::launch_grad_finish(h->tl, used, h->pnum, adjoint ? static_cast<float2*>(gPv) : nullptr,
                             h->gpos_part, h->N, adjoint ? gpos : nullptr, h->err_part,
                             h->err_part_n, loss, h->err_dpart, h->stream));
  return PTY_OK;
}
}  // namespace

int pty_loss(pty_handle* h, const void* O, const void* P, const float* pos, float delta,
             float* loss) {
  g_err.clear();
  return grad_run(h, O, P, pos, delta, loss, nullptr, nullptr, nullptr, false);
}

int pty_loss_grad(pty_handle* h, const void* O, const void* P, const float* pos, float delta,
                  float* loss, void* gO, void* gP, float* gpos) {
  g_err.clear();
  return grad_run(h, O, P, pos, delta, loss, gO, gP, gpos, true);
}

int pty_get_refine_gaps(pty_handle* h, float* dst, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (!dst) return fail(PTY_EINVAL, "null destination");
  CU(cudaMemcpyAsync(dst, h->gap, sizeof(float) * h->N, kind_out(mem_kind), h->stream));
  if (mem_kind == PTY_MEM_HOST) CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

int pty_run_groups(pty_handle* h, int g_begin, int g_end, const pty_rpie_params* p,
                   float* err_out) {
  g_err.clear();
  TRY(check_handle(h, true));
  TRY(check_params(p));
  TRY(regroup(h, p->max_group));
  const int G = (int)h->gptr.size() - 1;
  if (g_begin < 0 || g_end > G || g_begin > g_end)
    return fail(PTY_EINVAL, "group range [%d,%d) outside [0,%d)", g_begin, g_end, G);
  TRY(ensure_err_cap(h, 1));
  CU(cudaMemsetAsync(h->err_part, 0, sizeof(float) * h->err_part_n, h->stream));
  for (int g = g_begin; g < g_end; ++g) TRY(run_group(h, g, p));
  if (err_out) {
    CU(pty::launch_err_reduce(h->err_part, h->err_part_n, 0.0, h->sum_d, h->err_iter,
                              h->err_dpart, h->stream));
    CU(cudaMemcpyAsync(err_out, h->err_iter, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return PTY_OK;
}

int pty_get_groups(pty_handle* h, int* n_groups, int32_t* group_ptr, int32_t* group_pos) {
  g_err.clear();
  TRY(check_handle(h, true));
  if (!n_groups) return fail(PTY_EINVAL, "null n_groups");
  TRY(regroup(h, h->grouped_max < 0 ? 0 : h->grouped_max));
  *n_groups = (int)h->gptr.size() - 1;
  if (group_ptr) std::copy(h->gptr.begin(), h->gptr.end(), group_ptr);
  if (group_pos) std::copy(h->gpos.begin(), h->gpos.end(), group_pos);
  return PTY_OK;
}

#define PTY_COPY_OUT(NAME, FIELD, COUNT, T)                                         \
  int NAME(pty_handle* h, void* dst, int mem_kind) {                                \
    g_err.clear();                                                                  \
    TRY(check_handle(h, false));                                                    \
    TRY(check_mem_kind(mem_kind));                                                  \
    if (!dst) return fail(PTY_EINVAL, "null destination");                          \
    CU(cudaMemcpyAsync(dst, h->FIELD, sizeof(T) * (COUNT), kind_out(mem_kind), h->stream)); \
    if (mem_kind == PTY_MEM_HOST) TRY(check_tma_error(h)); /* synchronises */       \
    return PTY_OK;                                                                  \
  }

PTY_COPY_OUT(pty_get_object, O, (size_t)h->Hy * h->Hx, float2)
PTY_COPY_OUT(pty_get_probe, P, (size_t)h->M * h->W * h->W, float2)

int pty_get_positions(pty_handle* h, float* dst, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (!dst) return fail(PTY_EINVAL, "null destination");
  CU(cudaMemcpyAsync(dst, h->pos, sizeof(float) * 2 * h->N, kind_out(mem_kind), h->stream));
  if (mem_kind == PTY_MEM_HOST) CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

int pty_set_object(pty_handle* h, const void* src, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (!src) return fail(PTY_EINVAL, "null source");
  CU(cudaMemcpyAsync(h->O, src, sizeof(float2) * h->Hy * h->Hx, kind_in(mem_kind), h->stream));
  return finite_check(h, h->O, (size_t)2 * h->Hy * h->Hx, "object");
}

int pty_set_probe(pty_handle* h, const void* src, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (!src) return fail(PTY_EINVAL, "null source");
  const size_t n = (size_t)h->M * h->W * h->W;
  CU(cudaMemcpyAsync(h->P, src, sizeof(float2) * n, kind_in(mem_kind), h->stream));
  TRY(finite_check(h, h->P, 2 * n, "probe"));
  CU(pty::launch_pmax(h->tl, h->P, h->pmax_part, h->stream));
  return PTY_OK;
}

int pty_set_positions(pty_handle* h, const float* src, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (!src) return fail(PTY_EINVAL, "null source");
  std::vector<float> old = h->pos_h;
  h->pos_h.resize(2 * (size_t)h->N);
  CU(cudaMemcpyAsync(h->pos_h.data(), src, sizeof(float) * 2 * h->N,
                     mem_kind == PTY_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->groups_valid = false;
  const int rc = regroup(h, h->grouped_max < 0 ? 0 : h->grouped_max);
  if (rc != PTY_OK) {
    h->pos_h = old;
    h->groups_valid = false;
    return rc;
  }
  CU(cudaMemcpyAsync(h->pos, h->pos_h.data(), sizeof(float) * 2 * h->N, cudaMemcpyHostToDevice,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

int pty_get_adam_state(pty_handle* h, float* m, float* v, int* t, int* iter, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (m) CU(cudaMemcpyAsync(m, h->am, sizeof(float) * 2 * h->N, kind_out(mem_kind), h->stream));
  if (v) CU(cudaMemcpyAsync(v, h->av, sizeof(float) * 2 * h->N, kind_out(mem_kind), h->stream));
  if (t) *t = h->adam_t;
  if (iter) *iter = h->iter;
  CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

int pty_set_adam_state(pty_handle* h, const float* m, const float* v, int t, int iter,
                       int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, false));
  TRY(check_mem_kind(mem_kind));
  if (t < 0 || iter < 0) return fail(PTY_EINVAL, "negative Adam step or iteration count");
  if (m) CU(cudaMemcpyAsync(h->am, m, sizeof(float) * 2 * h->N, kind_in(mem_kind), h->stream));
  if (v) CU(cudaMemcpyAsync(h->av, v, sizeof(float) * 2 * h->N, kind_in(mem_kind), h->stream));
  h->adam_t = t;
  h->iter = iter;
  CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

int pty_model_intensities(pty_handle* h, float* dst, int mem_kind) {
  g_err.clear();
  TRY(check_handle(h, true));
  TRY(check_mem_kind(mem_kind));
  if (!dst) return fail(PTY_EINVAL, "null destination");
  TRY(regroup(h, h->grouped_max < 0 ? 0 : h->grouped_max));
  const size_t W2 = (size_t)h->W * h->W;
  float* out = dst;
  float* tmp = nullptr;
  if (mem_kind == PTY_MEM_HOST) {
    TRY(alloc_into(h, tmp, (size_t)h->N * W2));
    out = tmp;
  }
  int rc = PTY_OK;
  for (int c0 = 0; c0 < h->N && rc == PTY_OK; c0 += h->Qc) {
    const int nc = std::min(h->Qc, h->N - c0);
    cudaError_t e = pty::launch_rows_fwd_plain(h->tl, h->O, h->Hx, h->P, h->iota + c0,
                                               h->corners, nc, h->tw, h->scratch,
                                               h->omax_part, h->stream);
    if (e == cudaSuccess)
      e = pty::launch_cols_intensity(h->tl, h->scratch, h->iota + c0, nc, h->tw, h->inv_w, out,
                                     h->stream);
    if (e != cudaSuccess) rc = fail(PTY_ECUDA, "model intensity launch: %s", cudaGetErrorString(e));
  }
  if (rc == PTY_OK && tmp) {
    if (cudaMemcpyAsync(dst, tmp, sizeof(float) * h->N * W2, cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      rc = fail(PTY_ECUDA, "model intensity copy failed");
  }
  if (tmp) {
    cudaStreamSynchronize(h->stream);
    h->dfree(tmp);
  }
  return rc;
}

int pty_set_tiling(pty_handle* h, const pty_tiling* t) {
  g_err.clear();
  TRY(check_handle(h, false));
  if (!t) return fail(PTY_EINVAL, "null tiling");
  const int W = h->W, M = h->M, L = pty::lanes_per_line(W);
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (t->R && (!pow2(t->R) || W % t->R || M * t->R * L > 256))
    return fail(PTY_EINVAL, "rows per CTA R=%d invalid for W=%d, M=%d", t->R, W, M);
  if (t->CB && (!pow2(t->CB) || t->CB < 2 || t->CB > 16 || (W / 2) % t->CB || M * t->CB * L > 384))
    return fail(PTY_EINVAL, "columns per CTA CB=%d invalid for W=%d, M=%d", t->CB, W, M);
  if (t->ppc < 0 || t->ppc > 64) return fail(PTY_EINVAL, "patches per CTA %d", t->ppc);
  if (t->ppcb < 0 || t->ppcb > 64) return fail(PTY_EINVAL, "column patches per CTA %d", t->ppcb);
  pty::PatchGeo npg{};
  if (t->fused) {
    if (t->fused < 0 || t->fused > 8 || !pow2(t->fused))
      return fail(PTY_EINVAL, "fused slabs per mode S=%d: 1, 2, 4 or 8", t->fused);
    npg = pty::make_patch_geo(W, M, t->fused);
    if (npg.ncap < 1)
      return fail(PTY_EINVAL, "the fused patch kernel does not fit W=%d, M=%d, S=%d", W, M,
                  t->fused);
  }
  pty::Tiling nt = pty::make_tiling(W, M, false, 512, t->R, t->ppc, t->CB);
  if (t->ppcb > 0) nt.ppcb = t->ppcb;
  if (!pty::tiling_fits(nt)) return fail(PTY_EINVAL, "tiling exceeds the per-CTA limits");
  // the registration passes take the same geometry where it fits their extra
  // crop plane, and the same patches per chunk
  // (the extra plane can push the column pass past two CTAs per SM: halve
  // its column block until two fit)
  int cbr = t->CB;
  pty::Tiling nr = pty::make_tiling(W, M, true, 512, t->R, t->ppc, cbr);
  while (cbr > 2 && 2 * (nr.smB + 1024) > (size_t)pty::smem_per_sm()) {
    cbr /= 2;
    nr = pty::make_tiling(W, M, true, 512, t->R, t->ppc, cbr);
  }
  if (t->ppcb > 0) nr.ppcb = t->ppcb;
  if (!pty::tiling_fits(nr)) nr = h->tlr;
  const size_t W2 = (size_t)W * W;
  const size_t budget = t->scratch_bytes ? t->scratch_bytes : ((size_t)64 << 20);
  const int Qc = (int)std::min<size_t>((size_t)h->N, std::max<size_t>(1, budget / (W2 * M * sizeof(float2))));
  const int Qcr = Qc;
  // the differentiable form's chunk (M far-field planes and the crop
  // gradient per patch) under the same budget
  const int Qcg = (int)std::min<size_t>((size_t)h->N,
                                        std::max<size_t>(1, budget / (W2 * (M + 1) * sizeof(float2))));
  // grow the buffers whose size depends on the tiling
  // slots for this ppc and for the default ppc (4) the batched form uses
  const int ppc_min = std::min(std::min(nt.ppc, nr.ppc), 4);
  const int nslots = std::max((std::max(std::max(Qc, Qcr), Qcg) + ppc_min - 1) / ppc_min,
                              npg.ncap);  // the fused kernel: one slot per cluster
  const size_t scratch = std::max(std::max((size_t)Qc * M, (size_t)Qcr * nr.npl),
                                  (size_t)Qcg * (M + 1)) * W2;
  const size_t cur_scratch = std::max(std::max((size_t)h->Qc * M, (size_t)h->Qcr * h->tlr.npl),
                                      (size_t)h->Qcg * (M + 1)) * W2;
  CU(cudaStreamSynchronize(h->stream));
  if (scratch > cur_scratch) {
    h->dfree(h->scratch);
    h->scratch = nullptr;
    h->scratch_n = 0;
    TRY(alloc_into(h, h->scratch, scratch));
    h->scratch_n = scratch;
  }
  if (Qcr > h->Qcr) {
    h->dfree(h->cval); h->dfree(h->cidx);
    h->cval = nullptr; h->cidx = nullptr;
    TRY(alloc_into(h, h->cval, (size_t)Qcr * W));
    TRY(alloc_into(h, h->cidx, (size_t)Qcr * W));
    if (h->upart) {
      h->dfree(h->upart);
      h->upart = nullptr;
      TRY(alloc_into(h, h->upart, (size_t)Qcr * (W / 16) * h->rg.K * h->rg.K));
    }
  }
  if (nslots > h->nslots) {
    h->dfree(h->pnum); h->dfree(h->pden); h->dfree(h->osum);
    h->pnum = nullptr; h->pden = nullptr; h->osum = nullptr;
    TRY(alloc_into(h, h->pnum, (size_t)nslots * M * W2));
    TRY(alloc_into(h, h->pden, (size_t)nslots * W2));
    TRY(alloc_into(h, h->osum, (size_t)nslots));
    h->nslots = nslots;
  }
  const size_t omax_need = (size_t)std::max(Qc, Qcr) * (W / std::min(nt.R, nr.R));
  h->dfree(h->omax_part);
  h->omax_part = nullptr;
  TRY(alloc_into(h, h->omax_part, std::max(omax_need, (size_t)std::max(Qc, Qcr) * W)));
  h->tl = nt;
  h->tlr = nr;
  h->pg = npg;
  remap_scratch(h);
  h->Qc = Qc;
  h->Qcr = Qcr;
  h->Qcg = Qcg;
  h->err_part_n = (size_t)h->N * (W / nt.CB);
  ++h->epoch;
  CU(pty::set_smem_limits(h->tl));
  CU(pty::set_smem_limits(h->tlr));
  CU(pty::set_grad_smem(h->tl));
  pty::fill_residency(h->tl);
  pty::fill_residency(h->tlr);
  return PTY_OK;
}

int pty_get_tiling(pty_handle* h, pty_tiling* t) {
  g_err.clear();
  if (!h || !t) return fail(PTY_EINVAL, "null argument");
  t->R = h->tl.R;
  t->ppc = h->tl.ppc;
  t->CB = h->tl.CB;
  t->scratch_bytes = (size_t)h->Qc * h->M * h->W * h->W * sizeof(float2);
  t->ppcb = h->tl.ppcb;
  t->fused = h->pg.S > 0 ? h->pg.S : 0;
  return PTY_OK;
}

int pty_profile(pty_handle* h, int mode) {
  g_err.clear();
  if (!h) return fail(PTY_EINVAL, "null handle");
  if (mode != 0 && mode != 1) return fail(PTY_EINVAL, "profile mode %d", mode);
  h->prof_mode = mode;
  return PTY_OK;
}

int pty_debug_stall_copies(pty_handle* h, int on) {
  g_err.clear();
  TRY(check_handle(h, false));
  if (on != 0 && on != 1) return fail(PTY_EINVAL, "on=%d", on);
  CU(cudaMemcpyAsync(h->tma_err + 1, &on, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return PTY_OK;
}

int pty_get_stats(pty_handle* h, pty_stats* out, int reset) {
  g_err.clear();
  TRY(check_handle(h, false));
  if (!out) return fail(PTY_EINVAL, "null stats");
  CU(cudaStreamSynchronize(h->stream));
  h->drain();
  for (int k = 0; k < PTY_K_COUNT; ++k) {
    out->launches[k] = h->n_launch[k];
    out->ms[k] = h->ms[k];
  }
  out->patches = h->patches;
  if (reset) {
    for (int k = 0; k < PTY_K_COUNT; ++k) {
      h->n_launch[k] = 0;
      h->ms[k] = 0;
    }
    h->patches = 0;
  }
  return PTY_OK;
}

int pty_group_positions(const float* pos, int N, int W, int max_group, const int32_t* order,
                        int32_t* group_ptr, int32_t* group_pos, int* n_groups) {
  g_err.clear();
  if (!pos || !group_ptr || !group_pos || !n_groups) return fail(PTY_EINVAL, "null argument");
  if (N < 1 || W < 1 || max_group < 0) return fail(PTY_EINVAL, "bad size");
  if (order && !valid_perm(order, N)) return fail(PTY_EINVAL, "order is not a permutation");
  std::vector<int2> c(N);
  for (int j = 0; j < N; ++j) {
    const double y = pos[2 * j], x = pos[2 * j + 1];
    if (!std::isfinite(y) || !std::isfinite(x)) return fail(PTY_EDATA, "position %d not finite", j);
    c[j] = make_int2((int)std::floor(y + 0.5), (int)std::floor(x + 0.5));
  }
  std::vector<int> gptr, gpos;
  greedy_group(c, W, order, max_group, gptr, gpos);
  *n_groups = (int)gptr.size() - 1;
  std::copy(gptr.begin(), gptr.end(), group_ptr);
  std::copy(gpos.begin(), gpos.end(), group_pos);
  return PTY_OK;
}

int pty_hermitian_eig(int M, const double* A, double* w, double* V) {
  g_err.clear();
  if (!A || !w || !V) return fail(PTY_EINVAL, "null argument");
  if (M < 1 || M > 16) return fail(PTY_EINVAL, "M=%d outside 1..16", M);
  std::vector<std::complex<double>> a((size_t)M * M), v((size_t)M * M);
  for (size_t i = 0; i < a.size(); ++i) {
    if (!std::isfinite(A[2 * i]) || !std::isfinite(A[2 * i + 1]))
      return fail(PTY_EDATA, "matrix entry %zu not finite", i);
    a[i] = std::complex<double>(A[2 * i], A[2 * i + 1]);
  }
  if (pty::hermitian_eig(M, a.data(), w, v.data()) != 0) return fail(PTY_EINVAL, "eigensolver");
  for (size_t i = 0; i < v.size(); ++i) {
    V[2 * i] = v[i].real();
    V[2 * i + 1] = v[i].imag();
  }
  return PTY_OK;
}

int pty_orthogonalize_probe(pty_handle* h, double* power_out) {
  g_err.clear();
  TRY(check_handle(h, false));
  if (!h->has_data) return fail(PTY_ESTATE, "pty_set_data has not been called");
  const int M = h->M, WW = h->W * h->W;
  if (!h->modes_G) TRY(alloc_into(h, h->modes_G, (size_t)2 * M * M));  // double2 as 2 doubles
  if (!h->modes_V) TRY(alloc_into(h, h->modes_V, (size_t)M * M));
  CU(pty::launch_gram(h->P, M, WW, h->modes_G, h->stream));
  std::vector<double> g((size_t)2 * M * M);
  CU(cudaMemcpyAsync(g.data(), h->modes_G, sizeof(double) * g.size(), cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  std::vector<std::complex<double>> G((size_t)M * M), V((size_t)M * M);
  for (size_t i = 0; i < G.size(); ++i) {
    if (!std::isfinite(g[2 * i]) || !std::isfinite(g[2 * i + 1]))
      return fail(PTY_EDATA, "probe holds a non-finite value");
    G[i] = std::complex<double>(g[2 * i], g[2 * i + 1]);
  }
  std::vector<double> w(M);
  if (pty::hermitian_eig(M, G.data(), w.data(), V.data()) != 0)
    return fail(PTY_EINVAL, "eigensolver");
  std::vector<float2> vf((size_t)M * M);
  for (size_t i = 0; i < vf.size(); ++i)
    vf[i] = make_float2((float)V[i].real(), (float)V[i].imag());
  CU(cudaMemcpyAsync(h->modes_V, vf.data(), sizeof(float2) * vf.size(), cudaMemcpyHostToDevice,
                     h->stream));
  CU(pty::launch_mix(h->P, M, WW, h->modes_V, h->stream));
  CU(pty::launch_pmax(h->tl, h->P, h->pmax_part, h->stream));
  CU(cudaStreamSynchronize(h->stream));  // vf is host memory of this call
  if (power_out) std::copy(w.begin(), w.end(), power_out);
  return PTY_OK;
}

// ===================================================================== batch
struct pty_batch {
  std::vector<pty_handle*> hs;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream to capture the graph on
  int device = 0;
  pty::BatchProb* probs_d = nullptr;
  pty::BatchTask* tasks_d = nullptr;
  size_t tasks_cap = 0;
  unsigned* next_d = nullptr;
  unsigned* done_d = nullptr;
  int* error_d = nullptr;
  std::vector<unsigned> total;
  std::vector<int> status;
  int ntask = 0;
  cudaGraphExec_t gexec = nullptr;
  pty_batch_schedule sched{4, 2, 4, 2000, 0, -1};
  ~pty_batch() {
    if (stream) cudaStreamSynchronize(stream);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(probs_d);
    cudaFree(tasks_d);
    cudaFree(next_d);
    cudaFree(done_d);
    cudaFree(error_d);
    for (pty_handle* h : hs) pty_destroy(h);
  }
};

namespace {
void split_range(int n, int parts, std::vector<std::pair<int, int>>& out) {
  out.clear();
  parts = std::max(1, std::min(parts, n));
  for (int i = 0; i < parts; ++i) {
    const int a = (int)((long long)n * i / parts), b = (int)((long long)n * (i + 1) / parts);
    if (b > a) out.push_back({a, b});
  }
}
}  // namespace

int pty_batch_create(const pty_problem_desc* ds, int n, pty_batch** out) {
  g_err.clear();
  if (!ds || !out || n < 1) return fail(PTY_EINVAL, "bad batch arguments");
  *out = nullptr;
  pty_batch* b = new (std::nothrow) pty_batch();
  if (!b) return fail(PTY_ENOMEM, "host allocation failed");
  b->stream = static_cast<cudaStream_t>(ds[0].stream);
  for (int i = 0; i < n; ++i) {
    pty_problem_desc d = ds[i];
    d.stream = ds[0].stream;
    pty_handle* h = nullptr;
    const int rc = pty_init_problem(&d, &h);
    if (rc != PTY_OK) {
      std::string msg = g_err;
      delete b;
      return fail(rc, "problem %d: %s", i, msg.c_str());
    }
    b->hs.push_back(h);
  }
  cudaGetDevice(&b->device);
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&b->probs_d, sizeof(pty::BatchProb) * n) != cudaSuccess ||
      cudaMalloc(&b->next_d, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->done_d, sizeof(unsigned) * n) != cudaSuccess ||
      cudaMalloc(&b->error_d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(PTY_ENOMEM, "batch device allocation failed");
  }
  b->status.assign(n, PTY_OK);
  *out = b;
  return PTY_OK;
}

int pty_batch_problem(pty_batch* b, int i, pty_handle** h) {
  g_err.clear();
  if (!b || !h || i < 0 || i >= (int)b->hs.size()) return fail(PTY_EINVAL, "bad batch index");
  *h = b->hs[i];
  return PTY_OK;
}

int pty_batch_set_schedule(pty_batch* b, const pty_batch_schedule* s) {
  g_err.clear();
  if (!b || !s) return fail(PTY_EINVAL, "null argument");
  if (s->split_rows < 1 || s->split_cols < 1 || s->split_probe < 1 || s->timeout_ms < 1 ||
      s->ctas < 0 || s->stall_problem >= (int)b->hs.size())
    return fail(PTY_EINVAL, "bad schedule");
  b->sched = *s;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return PTY_OK;
}

int pty_batch_run(pty_batch* b, int n_iter, const pty_rpie_params* p) {
  g_err.clear();
  if (!b) return fail(PTY_EINVAL, "null batch");
  TRY(check_params(p));
  if (n_iter < 1) return fail(PTY_EINVAL, "n_iter < 1");
  CU(cudaSetDevice(b->device));
  const int n = (int)b->hs.size();
  std::vector<pty::BatchProb> probs(n);
  std::vector<std::vector<std::vector<pty::BatchTask>>> phases(n);
  size_t smem = 0;
  std::vector<std::pair<int, int>> rng;
  for (int i = 0; i < n; ++i) {
    pty_handle* h = b->hs[i];
    if (!h->has_data) return fail(PTY_ESTATE, "problem %d has no data", i);
    TRY(regroup(h, p->max_group));
    TRY(ensure_err_cap(h, n_iter));
    const pty::Tiling t = pty::make_tiling(h->W, h->M, false, 256);
    if (t.thrA > 256 || t.thrB > 256 || t.thrC > 256)
      return fail(PTY_EINVAL, "problem %d: W=%d with M=%d modes exceeds the batched CTA", i,
                  h->W, h->M);
    smem = std::max(smem, pty::batch_smem(t));
    pty::BatchProb& pb = probs[i];
    pb.W = h->W; pb.M = h->M; pb.N = h->N; pb.Hx = h->Hx;
    pb.R = t.R; pb.ppc = t.ppc; pb.CB = t.CB; pb.n_pmax = t.n_pmax;
    pb.inv_w = h->inv_w; pb.update_probe = p->update_probe; pb.a = upd_args(p);
    TRY(host_sum(h));
    pb.inv_sumI = h->sumI > 0 ? 1.0 / h->sumI : 0.0;
    pb.tw = h->tw; pb.O = h->O; pb.P = h->P; pb.I = h->I; pb.corners = h->corners;
    pb.gpos = h->gpos_d; pb.scratch = h->scratch; pb.pnum = h->pnum; pb.pden = h->pden;
    pb.osum = h->osum; pb.omax_part = h->omax_part; pb.err_part = h->err_part;
    pb.pmax_part = h->pmax_part; pb.err_iter = h->err_iter;
    pb.err_part_n = (size_t)h->N * (h->W / t.CB);
    auto& ph = phases[i];
    unsigned before = 0;
    auto add_phase = [&](std::vector<pty::BatchTask>&& v) {
      for (auto& tk : v) tk.need = before;
      before += (unsigned)v.size();
      ph.push_back(std::move(v));
    };
    const int G = (int)h->gptr.size() - 1;
    for (int it = 0; it < n_iter; ++it) {
      for (int g = 0; g < G; ++g) {
        const int ng = h->gptr[g + 1] - h->gptr[g];
        for (int c0 = 0; c0 < ng; c0 += h->Qc) {
          const int nc = std::min(h->Qc, ng - c0);
          const int off = h->gptr[g] + c0;
          const int py = (nc + t.ppc - 1) / t.ppc;
          for (int kind : {pty::BT_ROWS, pty::BT_COLS, pty::BT_ROWS_INV}) {
            std::vector<pty::BatchTask> v;
            const bool cols = kind == pty::BT_COLS;
            const int ny = cols ? nc : py;
            split_range(cols ? h->W / t.CB : h->W / t.R, cols ? b->sched.split_cols : b->sched.split_rows, rng);
            for (int y = 0; y < ny; ++y)
              for (auto& r : rng) {
                pty::BatchTask tk{};
                tk.prob = i; tk.kind = kind; tk.x0 = r.first; tk.x1 = r.second; tk.y = y;
                tk.ids_off = off; tk.npatch = nc; tk.flag = (kind == pty::BT_ROWS_INV && c0 > 0);
                v.push_back(tk);
              }
            add_phase(std::move(v));
          }
        }
        if (p->update_probe) {
          std::vector<pty::BatchTask> v;
          split_range(t.n_pmax, b->sched.split_probe, rng);
          const int used = (std::min(h->Qc, ng) + t.ppc - 1) / t.ppc;
          for (auto& r : rng) {
            pty::BatchTask tk{};
            tk.prob = i; tk.kind = pty::BT_PROBE; tk.x0 = r.first; tk.x1 = r.second; tk.flag = used;
            v.push_back(tk);
          }
          add_phase(std::move(v));
        }
      }
      std::vector<pty::BatchTask> v(1);
      v[0] = pty::BatchTask{};
      v[0].prob = i; v[0].kind = pty::BT_ERR; v[0].it = it;
      add_phase(std::move(v));
    }
    b->total.resize(n);
    b->total[i] = before;
  }
  // interleave the problems pass by pass
  std::vector<pty::BatchTask> tasks;
  size_t maxph = 0;
  for (auto& ph : phases) maxph = std::max(maxph, ph.size());
  for (size_t f = 0; f < maxph; ++f)
    for (int i = 0; i < n; ++i)
      if (f < phases[i].size()) tasks.insert(tasks.end(), phases[i][f].begin(), phases[i][f].end());
  if (b->sched.stall_problem >= 0) {
    // test hook: a dependency that can never be met, so that the bounded
    // wait runs out and reports PTY_ETIMEOUT instead of hanging
    for (auto it = tasks.rbegin(); it != tasks.rend(); ++it)
      if (it->prob == b->sched.stall_problem) {
        it->need = 0xffffffffu;
        break;
      }
  }
  b->ntask = (int)tasks.size();
  if (tasks.size() > b->tasks_cap) {
    CU(cudaStreamSynchronize(b->stream));
    cudaFree(b->tasks_d);
    b->tasks_d = nullptr;
    CU(cudaMalloc(&b->tasks_d, sizeof(pty::BatchTask) * tasks.size()));
    b->tasks_cap = tasks.size();
  }
  CU(cudaMemcpyAsync(b->tasks_d, tasks.data(), sizeof(pty::BatchTask) * tasks.size(),
                     cudaMemcpyHostToDevice, b->stream));
  CU(cudaMemcpyAsync(b->probs_d, probs.data(), sizeof(pty::BatchProb) * n, cudaMemcpyHostToDevice,
                     b->stream));
  int ctas = 0;
  CU(pty::batch_grid(smem, &ctas));
  if (b->sched.ctas > 0) ctas = std::min(ctas, b->sched.ctas);
  // one graph: reset the counters, then the persistent launch
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(b->next_d, 0, sizeof(unsigned), b->cap);
  cudaMemsetAsync(b->done_d, 0, sizeof(unsigned) * n, b->cap);
  cudaMemsetAsync(b->error_d, 0, sizeof(int), b->cap);
  cudaError_t le = pty::launch_batch(b->probs_d, b->tasks_d, b->ntask, b->next_d, b->done_d,
                                     b->error_d, (unsigned long long)b->sched.timeout_ms * 1000000ull,
                                     ctas, smem, b->cap);
  cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(PTY_ECUDA, "batch graph capture: %s / %s", cudaGetErrorString(le), cudaGetErrorString(ce));
  }
  cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(PTY_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  for (pty_handle* h : b->hs) ++h->n_launch[PTY_K_OTHER];
  CU(cudaGraphLaunch(b->gexec, b->stream));
  std::vector<unsigned> done(n);
  int err = 0;
  CU(cudaMemcpyAsync(done.data(), b->done_d, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, b->stream));
  CU(cudaMemcpyAsync(&err, b->error_d, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  int bad = 0;
  for (int i = 0; i < n; ++i) {
    b->status[i] = done[i] == b->total[i] ? PTY_OK : PTY_ETIMEOUT;
    if (b->status[i] != PTY_OK) ++bad;
    else b->hs[i]->iter += n_iter;
    b->hs[i]->patches += (long long)n_iter * b->hs[i]->N;
  }
  if (bad)
    return fail(PTY_ETIMEOUT, "%d problem(s) did not finish: a bounded wait gave up (first on problem %d)",
                bad, err - 1);
  return PTY_OK;
}

int pty_batch_status(pty_batch* b, int* per_problem) {
  g_err.clear();
  if (!b || !per_problem) return fail(PTY_EINVAL, "null argument");
  std::copy(b->status.begin(), b->status.end(), per_problem);
  return PTY_OK;
}

int pty_batch_destroy(pty_batch* b) {
  if (b) {
    cudaSetDevice(b->device);
    delete b;
  }
  return PTY_OK;
}

int pty_fft2(void* data, int W, int batch, int inverse, void* stream) {
  g_err.clear();
  if (!data || batch < 1) return fail(PTY_EINVAL, "bad argument");
  if (!pty::supported_W(W)) return fail(PTY_EINVAL, "unsupported W=%d", W);
  CU(pty::launch_fft2(data, W, batch, inverse, nullptr, static_cast<cudaStream_t>(stream)));
  return PTY_OK;
}

}  // extern "C"
