// Persistent batched form of the M-rPIE passes.  Compiled as relocatable
// device code: the per-pass task functions are real calls, each with its own
// register allocation (bodies in pty_passes.cuh).
#include "pty_passes.cuh"

#include <algorithm>

namespace pty {

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

// Not inlined: each pass of each pattern size keeps its own register
// allocation instead of one allocation for all of them inside the persistent
// kernel.
template <int W>
__device__ __noinline__ void batch_rows(const BatchProb& pb, const BatchTask& tk) {
  const int* ids = pb.gpos + tk.ids_off;
  for (int bx = tk.x0; bx < tk.x1; ++bx) {
    rows_fwd_body<W>(pb.O, pb.Hx, pb.P, pb.M, pb.R, pb.ppc, ids, pb.corners, tk.npatch, pb.tw,
                     pb.scratch, pb.omax_part, pb.M, 0, bx, tk.y);
    __syncthreads();
  }
}
template <int W, int CB>
__device__ __noinline__ void batch_cols(const BatchProb& pb, const BatchTask& tk) {
  const int* ids = pb.gpos + tk.ids_off;
  for (int bx = tk.x0; bx < tk.x1; ++bx) {
    cols_body<W, CB, false, false>(pb.scratch, pb.M, pb.I, ids, pb.tw, pb.inv_w, pb.a.eps,
                                   pb.err_part, pb.M, 1, tk.npatch, bx, tk.y);
    __syncthreads();
  }
}
template <int W>
__device__ __noinline__ void batch_rows_inv(const BatchProb& pb, const BatchTask& tk) {
  const int* ids = pb.gpos + tk.ids_off;
  for (int bx = tk.x0; bx < tk.x1; ++bx) {
    rows_inv_body<W, true>(pb.O, pb.Hx, pb.P, pb.M, pb.R, pb.ppc, ids, pb.corners, tk.npatch,
                     pb.scratch, pb.omax_part, pb.pmax_part, pb.n_pmax, pb.tw, pb.a, pb.pnum,
                     pb.pden, pb.osum, tk.flag, pb.M, 0, bx, tk.y);
    __syncthreads();
  }
}

template <int W>
__device__ __forceinline__ void batch_task(const BatchProb& pb, const BatchTask& tk) {
  switch (tk.kind) {
    case BT_ROWS:
      batch_rows<W>(pb, tk);
      break;
    case BT_COLS:
      if (pb.CB == 2) batch_cols<W, 2>(pb, tk);
      else if (pb.CB == 4) batch_cols<W, 4>(pb, tk);
      else if (pb.CB == 8) batch_cols<W, 8>(pb, tk);
      else batch_cols<W, 16>(pb, tk);
      break;
    case BT_ROWS_INV:
      batch_rows_inv<W>(pb, tk);
      break;
    case BT_PROBE:
      for (int bx = tk.x0; bx < tk.x1; ++bx) {
        probe_apply_body(pb.P, pb.M, W * W, pb.pnum, pb.pden, pb.osum, tk.flag, pb.a.alpha_P,
                         pb.a.reg_eps, pb.pmax_part, bx, pb.n_pmax);
        __syncthreads();
      }
      break;
    default:
      err_reduce_body(pb.err_part, pb.err_part_n, pb.inv_sumI, nullptr, pb.err_iter + tk.it);
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

size_t batch_smem(const Tiling& t) {
  // the batched column pass reads straight into registers: no stage
  const size_t smB = t.smB - (size_t)t.M * t.W * t.CB * sizeof(float2);
  return std::max({t.smA_staged, smB, t.smC, (size_t)256 * sizeof(double)});  // 256: the error reduction
}

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
