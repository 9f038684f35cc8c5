// Error state, FFT length factoring and a device-wide exclusive scan.
#include <atomic>
#include <string>

#include "common.cuh"

namespace vc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

static thread_local cudaStream_t g_alloc_stream = nullptr;
static bool g_pool_ready[128] = {false};

void set_alloc_stream(cudaStream_t s) {
  g_alloc_stream = s;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return;
  if (!g_pool_ready[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;       // keep freed blocks in this process's pool
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pool_ready[dev] = true;
  }
}
cudaStream_t alloc_stream() { return g_alloc_stream; }

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void adjust_launch_count(int64_t delta) { g_launches.fetch_add(delta, std::memory_order_relaxed); }

// Factor L into radices: 16, 8, 4, 2 for the powers of two, 9, 3, 5, 7 for
// the odd part; returns false if L has another prime factor.
bool factor_length(int L, int* radix, int* nst) {
  int n = 0;
  int r = L;
  if (L < 1) return false;
  // the power-of-two part 2^k in radices 16/8/4 without a radix-2 stage
  // unless k = 1: k = 4a + 1 becomes 16^(a-1) 8 4
  int k = 0;
  while (r % 2 == 0) { ++k; r /= 2; }
  if (k == 1) {
    radix[n++] = 2;
  } else if (k >= 2) {
    int a = k / 4;
    const int rem = k % 4;
    if (rem == 1) --a;
    for (int i = 0; i < a && n < kMaxStages; ++i) radix[n++] = 16;
    if (rem == 1 && n + 1 < kMaxStages) { radix[n++] = 8; radix[n++] = 4; }
    if (rem == 2 && n < kMaxStages) radix[n++] = 4;
    if (rem == 3 && n < kMaxStages) radix[n++] = 8;
  }
  while (r % 9 == 0 && n < kMaxStages) { radix[n++] = 9; r /= 9; }
  for (int p : {3, 5, 7})
    while (r % p == 0 && n < kMaxStages) { radix[n++] = p; r /= p; }
  *nst = n;
  return r == 1;
}

// Relative cost of transforming along an axis of padded length L: every
// stage is one shared-memory round trip plus its butterfly work, and two
// round trips' worth of memory traffic per point come on top.
double fft_cost(int L) {
  int rad[kMaxStages], nst = 0;
  if (!factor_length(L, rad, &nst)) return 1e300;
  double c = 2.0;
  for (int s = 0; s < nst; ++s) {
    switch (rad[s]) {
      case 2: c += 1.3; break;
      case 3: c += 1.5; break;
      case 4: c += 1.4; break;
      case 5: c += 1.8; break;
      case 7: c += 2.2; break;
      case 8: c += 1.6; break;
      case 9: c += 1.9; break;
      default: c += 1.8; break;   // 16
    }
  }
  return c * (double)L;
}

// ---------------------------------------------------------------- scan
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_incl_scan(int v, int* warp_sums) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += warp_sums[wid - 1];
  return v;
}

__global__ void scan_block_sums(const int32_t* __restrict__ d, int64_t n, int32_t* __restrict__ sums) {
  __shared__ int ws[32];
  int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int v = (i < n) ? d[i] : 0;
  int s = block_incl_scan(v, ws);
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = s;
}

// exclusive scan of sums[0..nb) in one block; total -> sums[nb]
__global__ void scan_sums_single(int32_t* sums, int64_t nb) {
  __shared__ int ws[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kScanBlock) {
    int64_t i = base + threadIdx.x;
    int v = (i < nb) ? sums[i] : 0;
    int s = block_incl_scan(v, ws);
    int c = carry;
    if (i < nb) sums[i] = c + s - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = c + s;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_apply(int32_t* __restrict__ d, int64_t n, const int32_t* __restrict__ sums) {
  __shared__ int ws[32];
  int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int v = (i < n) ? d[i] : 0;
  int s = block_incl_scan(v, ws);
  if (i < n) d[i] = sums[blockIdx.x] + s - v;
}

int64_t scan_tmp_elems(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

int exclusive_scan_i32(int32_t* data, int64_t n, int32_t* tmp, int64_t* total_host,
                       cudaStream_t st) {
  int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb == 0) {
    if (total_host) *total_host = 0;
    return VOXCAP_OK;
  }
  scan_block_sums<<<(unsigned)nb, kScanBlock, 0, st>>>(data, n, tmp); ::vc::note_launch();
  scan_sums_single<<<1, kScanBlock, 0, st>>>(tmp, nb); ::vc::note_launch();
  scan_apply<<<(unsigned)nb, kScanBlock, 0, st>>>(data, n, tmp); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  if (total_host) {
    int32_t t = 0;
    VC_CUDA(cudaMemcpyAsync(&t, tmp + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    *total_host = t;
  }
  return VOXCAP_OK;
}

}  // namespace vc
