// mgpbd_true_residual_noalloc: the FP64 true relative residual |b - A x| / |b|
// of an instance's level-0 matrix, computed without allocating any memory.
//
// Who needs it: code that must not call cudaMalloc while it runs -- a thread
// that is capturing a CUDA stream into a graph (allocation is not allowed
// during global-mode capture), a real-time loop that cannot stall on the
// allocator, or a host application whose device memory is owned by another
// pool.  Such a caller passes its own input and output buffers; the only
// other memory the kernel touches is a fixed block-partials array that lives
// in this file as a static device array.
//
// The array (kScratchBlocks x 2 doubles + a counter, about 1 MiB) is created
// when the library is loaded and is held by every GPU that loads the library
// until the process exits.  All calls share it and it keeps the last call's
// contents; the block counter that must start at zero is cleared before each
// launch.  Two calls that run at the same time on the GPU (different streams,
// or different host threads) use the same array and race: callers must
// serialise them.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture begins.
#include <mutex>
#include <string>

#include "common.cuh"

namespace mg {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocLanes = 4;                                   // lanes per row
constexpr int kNoAllocRowsPerBlock = kNoAllocThreads / kNoAllocLanes;  // 64
constexpr int kScratchBlocks = 65536;
constexpr int64_t kNoAllocMaxRows = (int64_t)kScratchBlocks * kNoAllocRowsPerBlock;

struct NoAllocScratch {
  double partials[2 * kScratchBlocks];  // per block: |b - A x|^2 and |b|^2
  unsigned int counter;
  unsigned int pad[63];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// one block per 64 rows, 4 lanes per row; the last block to finish folds the
// partials in block order and writes the relative residual
__global__ void k_true_resid_noalloc(int n, const int64_t *ptr, const int32_t *col,
                                     const double *val, const double *x, const double *b,
                                     NoAllocScratch *scr, double *out) {
  __shared__ double ws_r[kNoAllocThreads / 32], ws_b[kNoAllocThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = threadIdx.x & (kNoAllocLanes - 1);
  const int64_t i = (int64_t)blockIdx.x * kNoAllocRowsPerBlock + threadIdx.x / kNoAllocLanes;
  double s = 0.0;
  if (i < n)
    for (int64_t k = ptr[i] + g; k < ptr[i + 1]; k += kNoAllocLanes)
      s = fma(val[k], x[col[k]], s);
#pragma unroll
  for (int o = kNoAllocLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  double rr = 0.0, bb = 0.0;
  if (i < n && g == 0) {
    double ri = b[i] - s;
    rr = ri * ri;
    bb = b[i] * b[i];
  }
  rr = warp_sum(rr);
  bb = warp_sum(bb);
  if (lane == 0) {
    ws_r[wid] = rr;
    ws_b[wid] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, tb = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) {
      tr += ws_r[w];
      tb += ws_b[w];
    }
    scr->partials[2 * blockIdx.x] = tr;
    scr->partials[2 * blockIdx.x + 1] = tb;
    __threadfence();
    unsigned t = atomicAdd(&scr->counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tr = 0.0, tb = 0.0;
  for (int blk = threadIdx.x; blk < (int)gridDim.x; blk += blockDim.x) {
    tr += ((volatile double *)scr->partials)[2 * blk];
    tb += ((volatile double *)scr->partials)[2 * blk + 1];
  }
  tr = warp_sum(tr);
  tb = warp_sum(tb);
  if (lane == 0) {
    ws_r[wid] = tr;
    ws_b[wid] = tb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, sb = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) {
      sr += ws_r[w];
      sb += ws_b[w];
    }
    out[0] = sb > 0.0 ? sqrt(sr) / sqrt(sb) : 0.0;
    scr->counter = 0;
  }
}

// device address of the static array on device `dev`, looked up once per
// device (the caller has checked that `dev` is current)
static NoAllocScratch *scratch_for_device(int dev, mgpbd_status *st) {
  static std::mutex mu;
  static NoAllocScratch *addr[64] = {nullptr};
  if (dev < 0 || dev >= 64) {
    set_error("mgpbd_true_residual_noalloc: device ordinal above 63");
    *st = MGPBD_E_INVALID;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *st = cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress",
                      __FILE__, __LINE__);
      return nullptr;
    }
    addr[dev] = static_cast<NoAllocScratch *>(p);
  }
  *st = MGPBD_OK;
  return addr[dev];
}

}  // namespace mg

using namespace mg;

extern "C" mgpbd_status mgpbd_true_residual_noalloc(mgpbd_handle_t *hh, const double *d_b,
                                                    const double *d_x, double *d_out) {
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h || !d_b || !d_x || !d_out) {
    set_error("mgpbd_true_residual_noalloc: null argument");
    return MGPBD_E_INVALID;
  }
  const Level &L = h->lev[0];
  if ((int64_t)L.n > kNoAllocMaxRows) {
    set_error("mgpbd_true_residual_noalloc: the instance has more than 4,194,304 constraint "
              "rows, the limit of its static scratch (65,536 blocks of 64 rows)");
    return MGPBD_E_INVALID;
  }
  // the array's address is per device and the kernel runs on the instance's
  // stream, so the instance's device must be the current one
  int dev = -1;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) {
    set_error("mgpbd_true_residual_noalloc: the instance lives on device " +
              std::to_string(h->device) + " but device " + std::to_string(dev) +
              " is current; make the instance's device current first");
    return MGPBD_E_INVALID;
  }
  mgpbd_status st = MGPBD_OK;
  NoAllocScratch *scr = scratch_for_device(dev, &st);
  if (!scr) return st;
  if (L.n == 0) {
    MG_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), h->stream));
    return MGPBD_OK;
  }
  MG_CUDA(cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), h->stream));
  const int blocks = (int)((L.n + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock);
  k_true_resid_noalloc<<<blocks, kNoAllocThreads, 0, h->stream>>>(L.n, L.ptr, L.col, L.val, d_x,
                                                                   d_b, scr, d_out);
  MG_LAUNCH("k_true_resid_noalloc");
  return MGPBD_OK;
}
