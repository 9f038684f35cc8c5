// Tucker restoration of the Toeplitz tensors (Eq. 13, Sec. II.C):
//   X = S x1 U1 x2 U2 x3 U3,  X[i,j,k] = sum_abc S[a,b,c] U1[i,a] U2[j,b] U3[k,c],
// as three mode products, each a (batched) GEMM C = A B^T on the 5th-
// generation tensor cores (tcgen05.mma, kind::tf32, accumulators in TMEM).
//
// Precision: every FP64 operand x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi) and each product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation, which keeps
// about 21 mantissa bits -- below the Tucker truncation tolerances the
// restored tensors are used with (1e-6 ... 1e-4 relative, Sec. III.B).
//
// One CTA (4 warps) computes a 128 x 64 tile of C: operands are staged in
// shared memory in the canonical K-major layout without swizzle (8-row x
// 16-byte core matrices), one thread issues the MMAs, a tcgen05.commit
// arrives on an mbarrier, and the 4 warps read the accumulator lanes back
// with tcgen05.ld and store FP64.  Every wait on the mbarrier is bounded:
// on timeout the kernel records an error, releases its TMEM and returns.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace vc {

constexpr int kTM = 128;           // MMA M (TMEM lanes)
constexpr int kTN = 64;            // MMA N (TMEM columns)
constexpr int kKC = 32;            // K per shared-memory chunk (4 MMAs of K = 8)
constexpr int kTcThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 26;

struct GemmArgs {
  const double* A;   // A[b][m][k] = A[b*sAb + m*sAm + k*sAk]
  const double* B;   // B[b][n][k]
  double* C;         // C[b][m][n]
  int M, N, K, batch;
  int64_t sAb, sAm, sAk, sBb, sBn, sBk, sCb, sCm, sCn;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// byte offset of (row, k) in a K-major, no-swizzle tile with kKC columns:
// core matrices of 8 rows x 16 bytes; K-adjacent core matrices 128 B apart
// (leading byte offset), row-adjacent groups kKC/4 * 128 B apart (stride).
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * (kKC / 4) * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (kKC / 4) * 128;
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  return d;                          // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok;
}

__global__ void __launch_bounds__(kTcThreads) k_tc_gemm(GemmArgs g, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  // layout: A_hi, A_lo (kTM x kKC tf32 each), B_hi, B_lo (kTN x kKC), mbarrier, tmem slot
  unsigned char* a_hi = tsm;
  unsigned char* a_lo = a_hi + kTM * kKC * 4;
  unsigned char* b_hi = a_lo + kTM * kKC * 4;
  unsigned char* b_lo = b_hi + kTN * kKC * 4;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + kTN * kKC * 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN, b = blockIdx.z;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  // instruction descriptor: D = F32, A = B = TF32, both K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                         ((uint32_t)(kTM >> 4) << 24);
  uint32_t phase = 0;
  bool failed = false;
  const int nchunks = (g.K + kKC - 1) / kKC;
  for (int ch = 0; ch < nchunks && !failed; ++ch) {
    const int k0 = ch * kKC;
    // stage A and B (FP64 -> FP32 -> tf32 hi / lo), zero outside the matrices
    for (int t = threadIdx.x; t < kTM * kKC; t += kTcThreads) {
      int row, k;
      if (g.sAk == 1) { row = t / kKC; k = t % kKC; } else { row = t % kTM; k = t / kTM; }
      const int gm = m0 + row, gk = k0 + k;
      float v = 0.f;
      if (gm < g.M && gk < g.K) v = (float)g.A[(int64_t)b * g.sAb + (int64_t)gm * g.sAm + (int64_t)gk * g.sAk];
      const uint32_t hi = to_tf32(v);
      const uint32_t lo = to_tf32(v - __uint_as_float(hi));
      const uint32_t off = kmajor_off(row, k);
      *reinterpret_cast<uint32_t*>(a_hi + off) = hi;
      *reinterpret_cast<uint32_t*>(a_lo + off) = lo;
    }
    for (int t = threadIdx.x; t < kTN * kKC; t += kTcThreads) {
      int row, k;
      if (g.sBk == 1) { row = t / kKC; k = t % kKC; } else { row = t % kTN; k = t / kTN; }
      const int gn = n0 + row, gk = k0 + k;
      float v = 0.f;
      if (gn < g.N && gk < g.K) v = (float)g.B[(int64_t)b * g.sBb + (int64_t)gn * g.sBn + (int64_t)gk * g.sBk];
      const uint32_t hi = to_tf32(v);
      const uint32_t lo = to_tf32(v - __uint_as_float(hi));
      const uint32_t off = kmajor_off(row, k);
      *reinterpret_cast<uint32_t*>(b_hi + off) = hi;
      *reinterpret_cast<uint32_t*>(b_lo + off) = lo;
    }
    // make the generic-proxy shared-memory writes visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const unsigned char* As[3] = {a_hi, a_hi, a_lo};
      const unsigned char* Bs[3] = {b_hi, b_lo, b_hi};
      for (int term = 0; term < 3; ++term)
        for (int kk = 0; kk < kKC / 8; ++kk) {
          // K = 8 tf32 = two core matrices: advance by 2 x 128 B
          const uint64_t da = smem_desc(smem_u32(As[term]) + kk * 256);
          const uint64_t db = smem_desc(smem_u32(Bs[term]) + kk * 256);
          const uint32_t acc = (ch > 0 || term > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar)));
    }
    // every thread waits (bounded) for the MMAs of this chunk
    uint32_t ok = 0;
    for (uint32_t it = 0; it < kWaitLimit && !ok; ++it) ok = mbar_try_wait(smem_u32(mbar), phase);
    // one decision for the whole CTA, so that warp-wide tcgen05 instructions
    // below are executed by all lanes or by none
    if (__syncthreads_or(!ok)) {
      failed = true;
      if (threadIdx.x == 0) atomicExch(err, 1);
    }
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!failed) {
    // each warp reads its 32 TMEM lanes (rows), 16 columns at a time
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kTN; c0 += 16) {
      uint32_t r[16];
      const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
            "=r"(r[14]), "=r"(r[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < g.M)
        for (int q = 0; q < 16; ++q) {
          const int col = n0 + c0 + q;
          if (col < g.N)
            g.C[(int64_t)b * g.sCb + (int64_t)row * g.sCm + (int64_t)col * g.sCn] = (double)__uint_as_float(r[q]);
        }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN));
}

static int tc_gemm(const GemmArgs& g, int* err, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return VOXCAP_OK;
  const size_t sm = (size_t)(2 * kTM + 2 * kTN) * kKC * 4 + 64;
  VC_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  dim3 grid((g.M + kTM - 1) / kTM, (g.N + kTN - 1) / kTN, g.batch);
  k_tc_gemm<<<grid, kTcThreads, sm, st>>>(g, err); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

// X[i + D1 (j + D2 k)] = sum S[a][b][c] U1[i][a] U2[j][b] U3[k][c]
// S: r1 x r2 x r3 (c fastest); Un: Dn x rn row-major; all device pointers.
// T1 (r1 r2 D3) and T2 (r1 D3 D2) are scratch; a timed-out MMA wait sets
// *err.  Nothing is synchronised here.
static int tucker_expand_async(const double* S, int r1, int r2, int r3, const double* U1, int D1,
                               const double* U2, int D2, const double* U3, int D3, double* X, double* T1,
                               double* T2, int* err, cudaStream_t st) {
  GemmArgs g;
  // T1[a][b][k] = sum_c S[a][b][c] U3[k][c]
  g = GemmArgs{S, U3, T1, r1 * r2, D3, r3, 1, 0, r3, 1, 0, r3, 1, 0, D3, 1};
  VC_TRY(tc_gemm(g, err, st));
  // T2[a][k][j] = sum_b U2[j][b] T1[a][b][k]     (batch a)
  g = GemmArgs{U2, T1, T2, D2, D3, r2, r1, 0, r2, 1, (int64_t)r2 * D3, 1, D3, (int64_t)D3 * D2, 1, D2};
  VC_TRY(tc_gemm(g, err, st));
  // X[i + D1 n] = sum_a U1[i][a] T2[a][n],  n = j + D2 k
  g = GemmArgs{U1, T2, X, D1, D2 * D3, r1, 1, 0, r1, 1, 0, 1, (int64_t)D2 * D3, 0, 1, D1};
  VC_TRY(tc_gemm(g, err, st));
  return VOXCAP_OK;
}

// the same, standalone: its own scratch, one status read at the end
int tucker_expand(const double* S, int r1, int r2, int r3, const double* U1, int D1, const double* U2,
                  int D2, const double* U3, int D3, double* X, cudaStream_t st) {
  DBuf<double> T1, T2;
  DBuf<int> err;
  VC_TRY(T1.alloc((size_t)r1 * r2 * D3));
  VC_TRY(T2.alloc((size_t)r1 * D3 * D2));
  VC_TRY(err.alloc(1));
  VC_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  VC_TRY(tucker_expand_async(S, r1, r2, r3, U1, D1, U2, D2, U3, D3, X, T1.p, T2.p, err.p, st));
  int e = 0;
  VC_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  VC_CUDA(cudaStreamSynchronize(st));
  VC_CHECK(e == 0, VOXCAP_ERR_CUDA, "tensor-core Tucker expansion timed out waiting for its MMAs");
  return VOXCAP_OK;
}

void toeplitz_dims(const Geom& g, int kk, int* d);

// Restore the 15 Toeplitz tensors of the handle from Tucker factors of the
// four canonical tensors: each tensor is a canonical one with its modes
// mapped to the grid axes (test normal, source normal / in-plane axes) and
// cropped to the grid's offset ranges, so only the small core is permuted
// and the factor matrices are cut to their leading rows.
int build_toeplitz_tucker(Handle& h, const voxcap_tucker& tk) {
  // per tensor: canonical tensor t, grid axis of each of its modes
  int tsel[kNumKernels], axm[kNumKernels][3];
  size_t n1 = 1, n2 = 1, ncore = 1, nfac = 1;
  for (int kk = 0; kk < kNumKernels; ++kk) {
    int* d = h.tdims[kk];
    toeplitz_dims(h.g, kk, d);
    const int te = ker_test(kk), so = ker_src(kk);
    int* ax_of_mode = axm[kk];
    if (te == so) {
      tsel[kk] = kk >= 6 ? 1 : 0;
      ax_of_mode[0] = te;
      ax_of_mode[1] = te == 0 ? 1 : 0;
      ax_of_mode[2] = te == 2 ? 1 : 2;
    } else {
      tsel[kk] = kk >= 6 ? 3 : 2;
      ax_of_mode[0] = te;
      ax_of_mode[1] = so;
      ax_of_mode[2] = 3 - te - so;
    }
    const int t = tsel[kk];
    for (int m = 0; m < 3; ++m) {
      VC_CHECK(tk.dims[t][m] >= d[ax_of_mode[m]], VOXCAP_ERR_ARG,
               "Tucker tensor " + std::to_string(t) + " mode " + std::to_string(m) + " has " +
                   std::to_string(tk.dims[t][m]) + " rows, the grid needs " + std::to_string(d[ax_of_mode[m]]));
      VC_CHECK(tk.ranks[t][m] > 0 && tk.factor[t][m] != nullptr, VOXCAP_ERR_ARG, "bad Tucker factor");
    }
    VC_CHECK(tk.core[t] != nullptr, VOXCAP_ERR_ARG, "NULL Tucker core");
    int mode_of_ax[3];
    for (int m = 0; m < 3; ++m) mode_of_ax[ax_of_mode[m]] = m;
    const int* r = tk.ranks[t];
    const size_t rx = r[mode_of_ax[0]], ry = r[mode_of_ax[1]], rz = r[mode_of_ax[2]];
    n1 = std::max(n1, rx * ry * (size_t)d[2]);
    n2 = std::max(n2, rx * (size_t)d[2] * d[1]);
    ncore = std::max(ncore, rx * ry * rz);
    nfac = std::max(nfac, (size_t)d[0] * rx + (size_t)d[1] * ry + (size_t)d[2] * rz);
  }
  // scratch shared by the 15 restorations (stream-ordered), one status word
  DBuf<double> T1, T2, dcore, dfac;
  DBuf<int> err;
  VC_TRY(T1.alloc(n1));
  VC_TRY(T2.alloc(n2));
  VC_TRY(err.alloc(1));
  VC_TRY(dcore.alloc(ncore * kNumKernels));
  VC_TRY(dfac.alloc(nfac * kNumKernels));
  VC_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), h.stream));
  std::vector<double> core(ncore * kNumKernels);
  std::vector<double> fac(nfac * kNumKernels);
  for (int kk = 0; kk < kNumKernels; ++kk) {
    const int t = tsel[kk];
    const int* d = h.tdims[kk];
    int mode_of_ax[3];
    for (int m = 0; m < 3; ++m) mode_of_ax[axm[kk][m]] = m;
    const int* r = tk.ranks[t];
    const int rx = r[mode_of_ax[0]], ry = r[mode_of_ax[1]], rz = r[mode_of_ax[2]];
    // the core with its modes permuted to (x, y, z) grid axes
    double* cp = core.data() + ncore * kk;
    for (int p = 0; p < rx; ++p)
      for (int q = 0; q < ry; ++q)
        for (int s = 0; s < rz; ++s) {
          int idx[3];
          idx[mode_of_ax[0]] = p;
          idx[mode_of_ax[1]] = q;
          idx[mode_of_ax[2]] = s;
          cp[((size_t)p * ry + q) * rz + s] = tk.core[t][((size_t)idx[0] * r[1] + idx[1]) * r[2] + idx[2]];
        }
    // the factors' leading rows (the crop to the grid)
    double* fp = fac.data() + nfac * kk;
    size_t o = 0;
    for (int ax = 0; ax < 3; ++ax) {
      const int m = mode_of_ax[ax];
      const size_t n = (size_t)d[ax] * r[m];
      std::memcpy(fp + o, tk.factor[t][m], sizeof(double) * n);
      o += n;
    }
  }
  // two uploads, then the 15 expansions back to back
  VC_CUDA(cudaMemcpyAsync(dcore.p, core.data(), sizeof(double) * core.size(), cudaMemcpyHostToDevice, h.stream));
  VC_CUDA(cudaMemcpyAsync(dfac.p, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice, h.stream));
  for (int kk = 0; kk < kNumKernels; ++kk) {
    const int t = tsel[kk];
    const int* d = h.tdims[kk];
    int mode_of_ax[3];
    for (int m = 0; m < 3; ++m) mode_of_ax[axm[kk][m]] = m;
    const int* r = tk.ranks[t];
    const int rx = r[mode_of_ax[0]], ry = r[mode_of_ax[1]], rz = r[mode_of_ax[2]];
    const double* fp = dfac.p + nfac * kk;
    VC_TRY(h.toep[kk].alloc((size_t)d[0] * d[1] * d[2]));
    VC_TRY(tucker_expand_async(dcore.p + ncore * kk, rx, ry, rz, fp, d[0], fp + (size_t)d[0] * rx, d[1],
                               fp + (size_t)d[0] * rx + (size_t)d[1] * ry, d[2], h.toep[kk].p, T1.p, T2.p, err.p,
                               h.stream));
  }
  // one status read for the whole restoration: after a timed-out wait the
  // status is the only result to trust, and the set-up fails
  int e = 0;
  VC_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
  VC_CUDA(cudaStreamSynchronize(h.stream));
  VC_CHECK(e == 0, VOXCAP_ERR_CUDA, "tensor-core Tucker expansion timed out waiting for its MMAs");
  return VOXCAP_OK;
}

}  // namespace vc

extern "C" int voxcap_tucker_expand(const double* core, int r1, int r2, int r3, const double* U1, int D1,
                                    const double* U2, int D2, const double* U3, int D3, double* out) {
  using namespace vc;
  VC_CHECK(core && U1 && U2 && U3 && out, VOXCAP_ERR_ARG, "NULL array");
  VC_CHECK(r1 > 0 && r2 > 0 && r3 > 0 && D1 > 0 && D2 > 0 && D3 > 0, VOXCAP_ERR_ARG,
           "ranks and extents must be positive");
  set_alloc_stream(nullptr);
  return tucker_expand(core, r1, r2, r3, U1, D1, U2, D2, U3, D3, out, nullptr);
}
