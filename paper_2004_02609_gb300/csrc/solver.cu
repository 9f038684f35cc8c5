// Iterative solution (Sec. III: GMRES with restart 35) of the left-
// preconditioned system R A x = R b (Eq. 14), batched over right-hand sides,
// inside an FP64 iterative-refinement loop, and the capacitance matrix of
// Eq. 8.
//
// Arnoldi: classical Gram-Schmidt applied twice (CGS2) -- two fused
// dot/update sweeps over the Krylov basis per step instead of the j+1
// sequential sweeps of modified Gram-Schmidt, with at least its
// orthogonality.  Inner products and norms accumulate in FP64; the Hessenberg
// matrix, Givens rotations and residual estimates are FP64; the basis is
// stored in the inner solve's precision (FP32 for the refinement path).
//
// Refinement: r = b - A x in FP64 (FP64 product), inner GMRES on A d = r in
// FP32 (or FP64 for the plain path), x += d, until ||b - A x|| <= tol ||b||
// per column.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "internal.h"

namespace vc {

constexpr int kDotTB = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

// partial[col][i][chunk] = sum over the chunk of V_i[col] * w[col], i < nv
// (optionally first w -= sum_i coef[col][i] V_i[col]); with self_norm the one
// partial is ||w||^2 over the chunk.  The dot products of a sweep are spread
// over the warps of the block (warp q takes basis vectors q, q+8, ...).
template <typename T>
__global__ void k_gs_sweep(const T* __restrict__ V, T* __restrict__ w, int64_t N, int nrhs,
                           int nv_update, const double* __restrict__ coef, int coef_ld,
                           int nv_dot, bool self_norm, const int* __restrict__ active,
                           int nchunks, double* __restrict__ partial, int part_ld) {
  const int col = blockIdx.y;
  const int chunk = blockIdx.x;
  if (active && !active[col]) return;
  const int64_t per = (N + nchunks - 1) / nchunks;
  const int64_t lo = chunk * per, hi = min(N, lo + per);
  T* wc = w + (int64_t)col * N;
  const int64_t vstride = (int64_t)nrhs * N;
  if (nv_update > 0) {
    for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
      double acc = (double)wc[p];
      for (int i = 0; i < nv_update; ++i)
        acc -= coef[(int64_t)col * coef_ld + i] * (double)V[i * vstride + (int64_t)col * N + p];
      wc[p] = (T)acc;
    }
    __syncthreads();
  }
  const int nd = self_norm ? 1 : nv_dot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < nd; i += nw) {
    const T* vi = self_norm ? wc : V + i * vstride + (int64_t)col * N;
    double acc = 0.0;
    for (int64_t p = lo + lane; p < hi; p += 32) acc += (double)vi[p] * (double)wc[p];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) partial[((int64_t)col * part_ld + i) * nchunks + chunk] = acc;
  }
}

// out[col][i] (+)= sum_chunk partial[col][i][chunk]
__global__ void k_reduce_partial(const double* __restrict__ partial, int nchunks, int ni, int part_ld,
                                 const int* __restrict__ active, double* __restrict__ out, int out_ld,
                                 bool accumulate) {
  __shared__ double sh[32];
  const int col = blockIdx.y, i = blockIdx.x;
  if (active && !active[col]) return;
  double acc = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x)
    acc += partial[((int64_t)col * part_ld + i) * nchunks + c];
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    if (accumulate) out[(int64_t)col * out_ld + i] += s;
    else out[(int64_t)col * out_ld + i] = s;
  }
}

struct GState {      // per-column GMRES state, FP64, device
  double* H;         // [nrhs][m+1][m]  column-major in j: H[col][j*(m+1) + i]
  double* cs;        // [nrhs][m]
  double* sn;        // [nrhs][m]
  double* g;         // [nrhs][m+1]
  double* beta0;     // [nrhs] reference norm for the relative criterion
  double* hcol;      // [nrhs][m+1] current Arnoldi column (dots)
  double* hcol2;     // [nrhs][m+1] second-pass dots
  double* nrm2;      // [nrhs]
  int* active;       // [nrhs]
  int* kused;        // [nrhs] Arnoldi steps taken in the current cycle
  int* iters;        // [nrhs] total iterations
};

template <typename T>
__global__ void k_scale_cols(T* __restrict__ v, int64_t N, int nrhs, const double* __restrict__ f,
                             const int* __restrict__ mask) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int col = (int)(t / N);
  if (mask && !mask[col]) return;
  v[t] = (T)((double)v[t] * f[col]);
}

// start of a cycle: beta = ||V0||, g = beta e1, reference norm on the first cycle
__global__ void k_cycle_start(GState s, int nrhs, int m, bool first, double* inv_norm) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  double beta = sqrt(fmax(s.nrm2[col], 0.0));
  double* g = s.g + (int64_t)col * (m + 1);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  s.kused[col] = 0;
  if (first) {
    s.beta0[col] = beta;
    s.active[col] = beta > 0.0 ? 1 : 0;
    s.iters[col] = 0;
  }
  inv_norm[col] = beta > 0.0 ? 1.0 / beta : 0.0;
}

// after a cycle: a column is unconverged if its residual estimate is above
// rtol * beta0 and it has iterations left; mark it active for the next cycle
__global__ void k_reactivate(GState s, int nrhs, int m, const double* __restrict__ rtol, int max_it) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  const int k = s.kused[col];
  const double res = fabs(s.g[(int64_t)col * (m + 1) + k]);
  s.active[col] = (s.beta0[col] > 0.0 && res > rtol[col] * s.beta0[col] && s.iters[col] < max_it) ? 1 : 0;
}

// y = H^-1 g (upper triangular, k x k), stored in hcol
__global__ void k_backsolve(GState s, int nrhs, int m) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  const int k = s.kused[col];
  const double* H = s.H + (int64_t)col * (m + 1) * m;
  const double* g = s.g + (int64_t)col * (m + 1);
  double* y = s.hcol + (int64_t)col * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int c = i + 1; c < k; ++c) acc -= H[(int64_t)c * (m + 1) + i] * y[c];
    y[i] = H[(int64_t)i * (m + 1) + i] != 0.0 ? acc / H[(int64_t)i * (m + 1) + i] : 0.0;
  }
  for (int i = k; i <= m; ++i) y[i] = 0.0;
}

// x += sum_i y_i V_i
template <typename T>
__global__ void k_update_x(T* __restrict__ x, const T* __restrict__ V, int64_t N, int nrhs,
                           const double* __restrict__ y, const int* __restrict__ kused, int m) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int col = (int)(t / N);
  const int k = kused[col];
  double acc = (double)x[t];
  for (int i = 0; i < k; ++i) acc += y[(int64_t)col * (m + 1) + i] * (double)V[(int64_t)i * N * nrhs + t];
  x[t] = (T)acc;
}

template <typename T>
__global__ void k_sub(const T* __restrict__ b, const T* __restrict__ ax, T* __restrict__ r, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) r[t] = b[t] - ax[t];
}

// r = b - ax with ax from an FP32 product
__global__ void k_sub_f32(const double* __restrict__ b, const float* __restrict__ ax, double* __restrict__ r,
                          int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) r[t] = b[t] - (double)ax[t];
}

// r = b - ax in the columns whose mask is set; the others keep r
__global__ void k_sub_cols(const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ r,
                           int64_t N, int nrhs, const int* __restrict__ mask) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < N * nrhs && mask[t / N]) r[t] = b[t] - ax[t];
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (float)src[t];
}

__global__ void k_cast_scaled(const double* __restrict__ src, float* __restrict__ dst, int64_t N, int nrhs,
                              const double* __restrict__ f) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  dst[t] = (float)(src[t] * f[t / N]);
}

template <typename T>
__global__ void k_add_scaled(double* __restrict__ x, const T* __restrict__ d, int64_t N, int nrhs,
                             const double* __restrict__ f) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  x[t] += (double)d[t] * f[t / N];
}

// ------------------------------------------------------------------ GMRES
struct SolveCounters {
  int iters = 0;
  int matvecs = 0;
};

// chunks per column of the dot/update sweeps: at least one per 1024 rows,
// and for small systems enough (down to 128 rows each) for about one CTA per
// SM per column -- the FP64 inner products run at a low per-SM rate
// The count depends on N only, so a column's reductions are summed in the
// same order whatever other columns share its batch (a column's solve is
// bit-for-bit the same alone or batched; the sharded capacitance relies on it).
static int nchunks_for(int64_t N, int /*nrhs*/) {
  int64_t c = (N + 1023) / 1024;
  const int64_t fine = std::min<int64_t>((N + 127) / 128, 152);
  c = std::max(c, fine);
  if (c < 1) c = 1;
  if (c > 2048) c = 2048;
  return (int)c;
}

// ---- kernels of the graph-captured Arnoldi step (iteration index on the device) ----
// After the two Gram-Schmidt passes: H[:,j] = hcol + hcol2, h_{j+1,j} = sqrt(nrm2);
// Givens update; convergence test; scale factor for the new basis vector.
__device__ void givens_col(GState s, int col, int m, int j, double rtol, int max_it, double* inv_norm) {
  double* H = s.H + (int64_t)col * (m + 1) * m + (int64_t)j * (m + 1);
  double* cs = s.cs + (int64_t)col * m;
  double* sn = s.sn + (int64_t)col * m;
  double* g = s.g + (int64_t)col * (m + 1);
  for (int i = 0; i <= j; ++i) H[i] = s.hcol[(int64_t)col * (m + 1) + i] + s.hcol2[(int64_t)col * (m + 1) + i];
  double hn = sqrt(fmax(s.nrm2[col], 0.0));
  H[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * H[i] + sn[i] * H[i + 1];
    H[i + 1] = -sn[i] * H[i] + cs[i] * H[i + 1];
    H[i] = t;
  }
  double den = hypot(H[j], H[j + 1]);
  double c = den > 0.0 ? H[j] / den : 1.0;
  double sv = den > 0.0 ? H[j + 1] / den : 0.0;
  cs[j] = c;
  sn[j] = sv;
  H[j] = den;
  H[j + 1] = 0.0;
  g[j + 1] = -sv * g[j];
  g[j] = c * g[j];
  s.kused[col] = j + 1;
  s.iters[col] += 1;
  const bool conv = fabs(g[j + 1]) <= rtol * s.beta0[col];
  if (conv || hn == 0.0 || s.iters[col] >= max_it || j + 1 >= m) s.active[col] = 0;
  inv_norm[col] = hn > 0.0 ? 1.0 / hn : 0.0;
}

// True for the one CTA that finishes last among `count` (a fenced ticket; no
// CTA waits).  That CTA resets the ticket for the next use.
__device__ __forceinline__ bool last_cta(unsigned* ticket, unsigned count) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    is_last = atomicAdd(ticket, 1u) == count - 1;
    if (is_last) *ticket = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Control words of a restart cycle in device memory, written before each
// launch of the cycle graph (so the graph itself never changes).
struct CycleCtl {
  int max_it;         // iteration cap of the solve
  int steps;          // Arnoldi steps taken in this cycle (the loop guard)
};

struct StepArgs {
  int64_t N;
  int nrhs, m, nchunks, part_ld;
  CycleCtl* ctl;
  const double* rtol;   // [nrhs] inner relative tolerance of each column
  int* jdev;
  double* partial;
  unsigned* tickets;     // [nrhs] per-column tickets
  double* invn;
};

// One CGS pass of step j = *jdev over V[0..j] for column blockIdx.y, chunk
// blockIdx.x: pass 0: dots V_i . w -> hcol; pass 1: w -= sum hcol_i V_i, dots
// -> hcol2; pass 2: w -= sum hcol2_i V_i, ||w||^2 -> nrm2, then the Givens
// update of the column.  The last CTA of a column sums its partials.
// Arithmetic A of the update and of each lane's partial dot product: FP64
// (the method's orthogonalisation), or the FP32 basis's own precision under
// the fast refinement option (an FP32 basis is good to 6e-8 and a lane sums
// about 20 terms; FP64 arithmetic is 64 times slower on this GPU); FP64 from
// the lane sums on in both.
template <typename T, typename A>
__global__ void k_gs_step(const T* __restrict__ V, T* __restrict__ w, int pass, GState s, StepArgs a) {
  __shared__ double sh[32];
  __shared__ A cf[kMaxRestart + 1];
  const int col = blockIdx.y;
  const int chunk = blockIdx.x;
  if (!s.active[col]) return;                        // whole column: no CTA takes a ticket
  const int j = *a.jdev;
  const int nv = j + 1;
  const int64_t N = a.N;
  const int64_t per = (N + a.nchunks - 1) / a.nchunks;
  const int64_t lo = chunk * per, hi = min(N, lo + per);
  T* wc = w + (int64_t)col * N;
  const int64_t vstride = (int64_t)a.nrhs * N;
  if (pass > 0) {
    const double* coef = (pass == 1 ? s.hcol : s.hcol2) + (int64_t)col * (a.m + 1);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) cf[i] = (A)coef[i];
    __syncthreads();
    for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
      A acc = (A)wc[p];
      for (int i = 0; i < nv; ++i) acc -= cf[i] * (A)V[i * vstride + (int64_t)col * N + p];
      wc[p] = (T)acc;
    }
    __syncthreads();
  }
  const bool dot = pass < 2;
  const int nd = dot ? nv : 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < nd; i += nw) {
    const T* vi = dot ? V + i * vstride + (int64_t)col * N : wc;
    A lacc = 0;
    for (int64_t p = lo + lane; p < hi; p += 32) lacc += (A)vi[p] * (A)wc[p];
    double acc = (double)lacc;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) a.partial[((int64_t)col * a.part_ld + i) * a.nchunks + chunk] = acc;
  }
  if (!last_cta(a.tickets + col, (unsigned)a.nchunks)) return;
  double* out = pass == 0 ? s.hcol + (int64_t)col * (a.m + 1)
              : pass == 1 ? s.hcol2 + (int64_t)col * (a.m + 1) : s.nrm2 + col;
  for (int i = 0; i < nd; ++i) {
    double acc = 0.0;
    for (int c = threadIdx.x; c < a.nchunks; c += blockDim.x)
      acc += __ldcg(a.partial + ((int64_t)col * a.part_ld + i) * a.nchunks + c);
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) out[i] = t;
  }
  if (pass == 2 && threadIdx.x == 0 && j < a.m) givens_col(s, col, a.m, j, a.rtol[col], a.ctl->max_it, a.invn);
}

// V[j+1] = w * invn and vcur = V[j+1] for the columns that took step j; the
// columns' active flags to the host-mapped slot of step j's parity; the last
// CTA advances *jdev.
template <typename T>
__global__ void k_store_next(const T* __restrict__ w, T* __restrict__ V, T* __restrict__ vcur, GState s,
                             StepArgs a, unsigned* __restrict__ ticket, int* __restrict__ act_map) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int* jdev = a.jdev;
  const int j = *jdev;
  const int64_t N = a.N;
  if (t < N * a.nrhs && j < a.m) {
    const int col = (int)(t / N);
    if (s.kused[col] == j + 1) {          // this column took step j
      const T v = (T)((double)w[t] * a.invn[col]);
      V[(int64_t)(j + 1) * N * a.nrhs + t] = v;
      vcur[t] = v;
    }
  }
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < a.nrhs; c += blockDim.x) act_map[(j & 1) * a.nrhs + c] = s.active[c];
  if (last_cta(ticket, gridDim.x) && threadIdx.x == 0) *jdev = j + 1;
}

__global__ void k_cycle_ctl(CycleCtl* ctl, int max_it) {
  ctl->max_it = max_it;
  ctl->steps = 0;
}

// End of an Arnoldi step inside the cycle graph: run another step while some
// column is active, the cycle has steps left (*jdev < m) and the loop guard
// (steps counted here, independent of *jdev) has not reached m.
__global__ void k_loop_cond(cudaGraphConditionalHandle hc, CycleCtl* ctl, const int* __restrict__ jdev,
                            const int* __restrict__ active, int nrhs, int m) {
  if (threadIdx.x != 0) return;
  const int steps = ++ctl->steps;
  int any = 0;
  for (int c = 0; c < nrhs; ++c) any |= active[c];
  cudaGraphSetConditional(hc, (any && *jdev < m && steps < m) ? 1u : 0u);
}

// Solve R A d = R r (x0 = 0) per column to a preconditioned relative
// residual rtol_host[col] (host, one per column).  r, d: device [nrhs][N] in T.
// `adjoint`: use A^T.  A restart cycle is one launch of a CUDA graph: the host prepares the
// cycle's first basis vector, writes the cycle's control words, and launches
// the graph, whose conditional while node runs Arnoldi steps (product,
// preconditioner, two Gram-Schmidt passes with the Givens update, next basis
// vector, loop condition) on the device until every column has converged or
// the cycle is full; the host synchronises once per cycle, after the update
// of d.  The graph is instantiated once per handle, shape and precision.
template <typename T>
static int gmres(Handle& h, const T* r, T* d, int nrhs, const double* rtol_host, int max_it, bool adjoint,
                 SolveCounters* cnt) {
  const int64_t N = h.pan.N;
  const int m = std::max(1, h.opts.restart);
  cudaStream_t st = h.stream;
  const int nch = nchunks_for(N, nrhs);
  const size_t nV = (size_t)(m + 1) * nrhs * N;
  const size_t nW = (size_t)nrhs * N;
  size_t bytes = sizeof(T) * (nV + 3 * nW) + 256;
  const size_t nd_H = (size_t)nrhs * (m + 1) * m, nd_cs = (size_t)nrhs * m, nd_g = (size_t)nrhs * (m + 1);
  const size_t ndbl = nd_H + 2 * nd_cs + 3 * nd_g + 3 * (size_t)nrhs + (size_t)nrhs * (m + 1) * nch;
  bytes += sizeof(double) * ndbl + sizeof(int) * (3 * nrhs + 4) + sizeof(unsigned) * (nrhs + 1) + 256 +
           sizeof(CycleCtl) + sizeof(double) * nrhs + 64;
  VC_TRY(h.solver_ws.alloc(bytes));
  char* wp = h.solver_ws.p;
  T* V = reinterpret_cast<T*>(wp); wp += sizeof(T) * nV;
  T* W = reinterpret_cast<T*>(wp); wp += sizeof(T) * nW;
  T* W2 = reinterpret_cast<T*>(wp); wp += sizeof(T) * nW;
  T* vcur = reinterpret_cast<T*>(wp); wp += sizeof(T) * nW;
  wp = reinterpret_cast<char*>(((uintptr_t)wp + 15) & ~(uintptr_t)15);
  double* dp = reinterpret_cast<double*>(wp);
  GState s;
  s.H = dp; dp += nd_H;
  s.cs = dp; dp += nd_cs;
  s.sn = dp; dp += nd_cs;
  s.g = dp; dp += nd_g;
  s.hcol = dp; dp += nd_g;
  s.hcol2 = dp; dp += nd_g;
  s.beta0 = dp; dp += nrhs;
  s.nrm2 = dp; dp += nrhs;
  double* invn = dp; dp += nrhs;
  double* partial = dp; dp += (size_t)nrhs * (m + 1) * nch;
  int* ip = reinterpret_cast<int*>(dp);
  s.active = ip; ip += nrhs;
  s.kused = ip; ip += nrhs;
  s.iters = ip; ip += nrhs;
  int* jdev = ip; ip += 1;
  unsigned* tickets = reinterpret_cast<unsigned*>(ip + 1);    // [nrhs] columns, [nrhs] the store
  CycleCtl* ctl = reinterpret_cast<CycleCtl*>(((uintptr_t)(tickets + nrhs + 1) + 15) & ~(uintptr_t)15);
  double* rtol = reinterpret_cast<double*>(((uintptr_t)(ctl + 1) + 15) & ~(uintptr_t)15);
  VC_CUDA(cudaMemcpyAsync(rtol, rtol_host, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
  VC_CUDA(cudaMemsetAsync(d, 0, sizeof(T) * nW, st));
  VC_CUDA(cudaMemsetAsync(tickets, 0, sizeof(unsigned) * (nrhs + 1), st));
  VC_TRY(h.act_map.ensure((size_t)4 * nrhs));
  const int TB = 256;
  const unsigned gN = (unsigned)((N * nrhs + TB - 1) / TB);
  const unsigned gC = (unsigned)((nrhs + 63) / 64);
  // the product's tables and workspace must exist before capture (no
  // allocation or symbol copy inside the graph)
  VC_TRY(mvm_prepare(h, nrhs, sizeof(C_t<T>)));

  // ---- the restart-cycle graph, built once per key ----
  const bool fastgs = sizeof(T) == 4 && h.opts.fast_refine != 0;
  const uintptr_t key[10] = {sizeof(T) + (fastgs ? 16 : 0), (uintptr_t)adjoint, (uintptr_t)nrhs, (uintptr_t)N,
                             (uintptr_t)m,
                             (uintptr_t)h.solver_ws.p, (uintptr_t)h.ws.p,
                             (uintptr_t)(h.path + 2) |
                                 ((uintptr_t)(h.yvar[0] + 2 * h.yvar[1] + 4 * h.zfvar) << 8) |
                                 ((uintptr_t)h.zvar << 16) | ((uintptr_t)(h.ztx + 2) << 24),
                             (uintptr_t)(h.ytx[0] + 2) | ((uintptr_t)(h.ytx[1] + 2) << 8), (uintptr_t)h.act_map.d};
  bool same = h.gm.exec != nullptr;
  for (int i = 0; same && i < 10; ++i) same = h.gm.key[i] == key[i];
  if (!same) {
    h.gm.reset();
    const int64_t launches_before_capture = launch_count();
    cudaGraph_t graph = nullptr;
    int rc = cudaGraphCreate(&graph, 0) == cudaSuccess ? VOXCAP_OK : VOXCAP_ERR_CUDA;
    cudaGraphConditionalHandle hc = 0;
    cudaGraph_t body = nullptr;
    if (rc == VOXCAP_OK &&
        cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
      rc = VOXCAP_ERR_CUDA;
    if (rc == VOXCAP_OK) {
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = hc;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t wn;
      if (cudaGraphAddNode(&wn, graph, nullptr, nullptr, 0, &np) != cudaSuccess) rc = VOXCAP_ERR_CUDA;
      else body = np.conditional.phGraph_out[0];
    }
    cudaStream_t cap = nullptr;
    if (rc == VOXCAP_OK && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
      rc = VOXCAP_ERR_CUDA;
    if (rc == VOXCAP_OK) {
      const cudaStream_t saved = h.stream;
      h.stream = cap;
      if (cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
          cudaSuccess)
        rc = VOXCAP_ERR_CUDA;
      if (rc == VOXCAP_OK) rc = mvm<T>(h, vcur, W, nrhs, adjoint, nullptr);
      if (rc == VOXCAP_OK) rc = precond_apply<T>(h, W, W2, nrhs);
      if (rc == VOXCAP_OK) {
        dim3 gsw(nch, nrhs);
        StepArgs sa;
        sa.N = N; sa.nrhs = nrhs; sa.m = m; sa.nchunks = nch; sa.part_ld = m + 1;
        sa.ctl = ctl; sa.rtol = rtol; sa.jdev = jdev; sa.partial = partial;
        sa.tickets = tickets; sa.invn = invn;
        if (fastgs) {
          k_gs_step<T, T><<<gsw, kDotTB, 0, cap>>>(V, W2, 0, s, sa);
          k_gs_step<T, T><<<gsw, kDotTB, 0, cap>>>(V, W2, 1, s, sa);
          k_gs_step<T, T><<<gsw, kDotTB, 0, cap>>>(V, W2, 2, s, sa);
        } else {
          k_gs_step<T, double><<<gsw, kDotTB, 0, cap>>>(V, W2, 0, s, sa);
          k_gs_step<T, double><<<gsw, kDotTB, 0, cap>>>(V, W2, 1, s, sa);
          k_gs_step<T, double><<<gsw, kDotTB, 0, cap>>>(V, W2, 2, s, sa);
        }
        k_store_next<T><<<gN, TB, 0, cap>>>(W2, V, vcur, s, sa, tickets + nrhs, h.act_map.d);
        k_loop_cond<<<1, 32, 0, cap>>>(hc, ctl, jdev, s.active, nrhs, m);
      }
      cudaGraph_t captured = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(cap, &captured);
      h.stream = saved;
      if (rc == VOXCAP_OK && ce != cudaSuccess) rc = VOXCAP_ERR_CUDA;
    }
    if (cap) cudaStreamDestroy(cap);
    cudaGraphExec_t exec = nullptr;
    if (rc == VOXCAP_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = VOXCAP_ERR_CUDA;
    adjust_launch_count(launches_before_capture - launch_count());   // capture issued no launch
    if (rc != VOXCAP_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      const cudaError_t e = cudaGetLastError();
      set_error(std::string("building the GMRES cycle graph failed: ") + cudaGetErrorString(e));
      return VOXCAP_ERR_CUDA;
    }
    h.gm.graph = graph;
    h.gm.exec = exec;
    for (int i = 0; i < 10; ++i) h.gm.key[i] = key[i];
  }
  // kernel launches inside one Arnoldi step of the graph (counted per step run)
  const int step_launches = 5 + ((h.pre.kind == VOXCAP_PRECOND_BDD || h.pre.kind == VOXCAP_PRECOND_BD) &&
                                 h.pre.nblocks > 0 && h.pre.max_n > 0 ? 2 : 1) + 5;

  bool first = true;
  int total_it = 0;
  for (int cycle = 0; cycle < 100000; ++cycle) {
    // V0 = R (r - A d), vcur = V0 / ||V0||, j = 0
    if (first) {
      VC_TRY(precond_apply<T>(h, r, V, nrhs));
    } else {
      VC_TRY(mvm<T>(h, d, W, nrhs, adjoint, nullptr));
      cnt->matvecs += 1;
      k_sub<T><<<gN, TB, 0, st>>>(r, W, W2, N * nrhs); ::vc::note_launch();
      VC_TRY(precond_apply<T>(h, W2, V, nrhs));
    }
    dim3 gsw(nch, nrhs);
    k_gs_sweep<T><<<gsw, kDotTB, 0, st>>>(V, V, N, nrhs, 0, nullptr, 0, 0, true, nullptr, nch, partial, m + 1); ::vc::note_launch();
    k_reduce_partial<<<dim3(1, nrhs), kDotTB, 0, st>>>(partial, nch, 1, m + 1, nullptr, s.nrm2, 1, false); ::vc::note_launch();
    k_cycle_start<<<gC, 64, 0, st>>>(s, nrhs, m, first, invn); ::vc::note_launch();
    k_scale_cols<T><<<gN, TB, 0, st>>>(V, N, nrhs, invn, nullptr); ::vc::note_launch();
    VC_CUDA(cudaMemcpyAsync(vcur, V, sizeof(T) * nW, cudaMemcpyDeviceToDevice, st));
    VC_CUDA(cudaMemsetAsync(jdev, 0, sizeof(int), st));
    k_cycle_ctl<<<1, 1, 0, st>>>(ctl, max_it); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
    first = false;
    // the Arnoldi steps of the cycle run on the device
    VC_CUDA(cudaGraphLaunch(h.gm.exec, st));
    k_backsolve<<<gC, 64, 0, st>>>(s, nrhs, m); ::vc::note_launch();
    k_update_x<T><<<gN, TB, 0, st>>>(d, V, N, nrhs, s.hcol, s.kused, m); ::vc::note_launch();
    // a column that stopped only because the cycle ended is still unconverged:
    // re-activate it from the residual estimate (converged ones stay inactive)
    k_reactivate<<<gC, 64, 0, st>>>(s, nrhs, m, rtol, max_it); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
    // steps taken, iteration counts and active flags in one read-back
    // (mapped pinned host memory): the one synchronisation of the cycle
    int* its_h = h.act_map.h + 2 * nrhs;
    int* act_h = h.act_map.h + 3 * nrhs;
    int steps_h = 0;
    VC_CUDA(cudaMemcpyAsync(its_h, s.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaMemcpyAsync(act_h, s.active, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaMemcpyAsync(&steps_h, &ctl->steps, sizeof(int), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < steps_h * step_launches; ++q) ::vc::note_launch();
    cnt->matvecs += steps_h;
    total_it += steps_h;
    int maxit = 0;
    bool any = false;
    for (int c = 0; c < nrhs; ++c) {
      maxit = std::max(maxit, its_h[c]);
      any = any || act_h[c];
    }
    if (!any || maxit >= max_it) break;
  }
  cnt->iters += total_it;
  return VOXCAP_OK;
}

// column norms of a double [nrhs][N] array -> host
static int col_norms(Handle& h, const double* v, int nrhs, std::vector<double>& out, double* partial_ws,
                     double* dev_out) {
  const int64_t N = h.pan.N;
  const int nch = nchunks_for(N, nrhs);
  dim3 g(nch, nrhs);
  k_gs_sweep<double><<<g, kDotTB, 0, h.stream>>>(nullptr, const_cast<double*>(v), N, nrhs, 0, nullptr, 0,
                                                 0, true, nullptr, nch, partial_ws, 1); ::vc::note_launch();
  k_reduce_partial<<<dim3(1, nrhs), kDotTB, 0, h.stream>>>(partial_ws, nch, 1, 1, nullptr, dev_out, 1, false); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  out.resize(nrhs);
  VC_CUDA(cudaMemcpyAsync(out.data(), dev_out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, h.stream));
  VC_CUDA(cudaStreamSynchronize(h.stream));
  for (auto& x : out) x = std::sqrt(std::max(x, 0.0));
  return VOXCAP_OK;
}

int solve(Handle& h, const double* B, int nrhs, double tol, double* X, voxcap_stats* st, bool adjoint) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t N = h.pan.N;
  const bool refine = h.opts.precision == VOXCAP_FP32_REFINE;
  cudaStream_t s = h.stream;
  voxcap_stats loc = {};
  if (N == 0 || nrhs <= 0) {
    if (st) { *st = loc; st->converged = 1; }
    return VOXCAP_OK;
  }
  DBuf<double> R64, AX, dpart, dnorm, fac;
  DBuf<int> cmask;
  DBuf<float> rf, df;
  DBuf<double> d64;
  const size_t n = (size_t)N * nrhs;
  VC_TRY(R64.alloc(n));
  VC_TRY(AX.alloc(n));
  VC_TRY(dpart.alloc((size_t)nrhs * nchunks_for(N, nrhs) + 1));
  VC_TRY(dnorm.alloc(nrhs));
  VC_TRY(fac.alloc(nrhs));
  VC_TRY(cmask.alloc(nrhs));
  if (refine) { VC_TRY(rf.alloc(n)); VC_TRY(df.alloc(n)); }
  else VC_TRY(d64.alloc(n));
  std::vector<double> bn, rn;
  VC_TRY(col_norms(h, B, nrhs, bn, dpart.p, dnorm.p));
  VC_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * n, s));
  const int TB = 256;
  const unsigned gN = (unsigned)((n + TB - 1) / TB);
  SolveCounters cnt;
  const int max_sweeps = std::max(1, h.opts.max_sweeps);
  double worst = 0.0;
  bool conv = false;
  int sweeps = 0;
  // Under refinement with the fast option, the residual of a column whose
  // last sweep only had to reach a large residual (expected relative residual
  // >= 1e-5) is formed with an FP32 product: its error (~1e-7 of |b|) is two orders below that
  // residual, so the next correction is as good as with an FP64 residual.
  // Convergence is only ever decided on an FP64 residual, and each column's
  // choice depends on its own history only (products are column by column).
  std::vector<int> use32(nrhs, 0), need64(nrhs, 1);
  for (int sw = 0; sw <= max_sweeps; ++sw) {
    if (sw == 0) {
      VC_CUDA(cudaMemcpyAsync(R64.p, B, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      rn = bn;                                       // the first residual is B itself
    } else {
      bool any32 = false, any64 = false;
      for (int c = 0; c < nrhs; ++c) {
        need64[c] = !use32[c];
        any32 = any32 || use32[c];
      }
      if (any32) {
        k_to_f32<<<gN, TB, 0, s>>>(X, rf.p, (int64_t)n); ::vc::note_launch();
        VC_TRY(mvm<float>(h, rf.p, df.p, nrhs, adjoint, nullptr));
        cnt.matvecs += 1;
        k_sub_f32<<<gN, TB, 0, s>>>(B, df.p, R64.p, (int64_t)n); ::vc::note_launch();
        VC_CUDA(cudaGetLastError());
        VC_TRY(col_norms(h, R64.p, nrhs, rn, dpart.p, dnorm.p));
        for (int c = 0; c < nrhs; ++c)               // close to the end: decide on FP64
          if (use32[c] && bn[c] > 0.0 && rn[c] <= 10.0 * tol * bn[c]) need64[c] = 1;
      }
      for (int c = 0; c < nrhs; ++c) any64 = any64 || need64[c];
      if (any64) {
        VC_TRY(mvm<double>(h, X, AX.p, nrhs, adjoint, nullptr));
        cnt.matvecs += 1;
        if (any32) {
          VC_CUDA(cudaMemcpyAsync(cmask.p, need64.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
          k_sub_cols<<<gN, TB, 0, s>>>(B, AX.p, R64.p, N, nrhs, cmask.p); ::vc::note_launch();
        } else {
          k_sub<double><<<gN, TB, 0, s>>>(B, AX.p, R64.p, (int64_t)n); ::vc::note_launch();
        }
        VC_CUDA(cudaGetLastError());
        VC_TRY(col_norms(h, R64.p, nrhs, rn, dpart.p, dnorm.p));
      }
    }
    worst = 0.0;
    std::vector<double> f(nrhs), finv(nrhs), itol(nrhs);
    for (int c = 0; c < nrhs; ++c) {
      double rel = bn[c] > 0.0 ? rn[c] / bn[c] : 0.0;
      worst = std::max(worst, rel);
      // columns that already meet tol get a zero right-hand side
      bool done = rel <= tol || rn[c] == 0.0;
      f[c] = done ? 0.0 : 1.0 / rn[c];
      finv[c] = done ? 0.0 : rn[c];
      // inner tolerance of the column (its own, so that a column's solve does
      // not depend on the others in the batch).  Plain FP64: aim to finish in
      // this sweep.  FP32 inside refinement: a sweep reduces the residual by
      // inner_tol at most (FP32 GMRES stagnates when pushed much further,
      // and its Krylov space is rebuilt each sweep anyway) and by no more
      // than finishing needs, so the last sweep does not over-solve
      const double need = done ? 1.0 : tol / rel;
      itol[c] = refine ? std::max(5e-6, std::max(h.opts.inner_tol, 0.5 * need))
                       : std::min(1e-2, std::max(1e-14, 0.5 * need));
    }
    if (worst <= tol) { conv = true; break; }
    if (sw == max_sweeps || cnt.iters >= h.opts.max_iters) break;
    ++sweeps;
    for (int c = 0; c < nrhs; ++c) {
      const double rel = bn[c] > 0.0 ? rn[c] / bn[c] : 0.0;
      use32[c] = refine && h.opts.fast_refine && f[c] != 0.0 && rel * itol[c] >= 1e-5;
    }
    int left = std::max(1, h.opts.max_iters - cnt.iters);
    VC_CUDA(cudaMemcpyAsync(fac.p, f.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    if (refine) {
      k_cast_scaled<<<gN, TB, 0, s>>>(R64.p, rf.p, N, nrhs, fac.p); ::vc::note_launch();
      VC_TRY(gmres<float>(h, rf.p, df.p, nrhs, itol.data(), left, adjoint, &cnt));
      VC_CUDA(cudaMemcpyAsync(fac.p, finv.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      k_add_scaled<float><<<gN, TB, 0, s>>>(X, df.p, N, nrhs, fac.p); ::vc::note_launch();
    } else {
      // scale the FP64 residual to unit norm too (keeps the criterion relative)
      k_scale_cols<double><<<gN, TB, 0, s>>>(R64.p, N, nrhs, fac.p, nullptr); ::vc::note_launch();
      VC_TRY(gmres<double>(h, R64.p, d64.p, nrhs, itol.data(), left, adjoint, &cnt));
      VC_CUDA(cudaMemcpyAsync(fac.p, finv.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      k_add_scaled<double><<<gN, TB, 0, s>>>(X, d64.p, N, nrhs, fac.p); ::vc::note_launch();
    }
    VC_CUDA(cudaGetLastError());
  }
  VC_CUDA(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  loc.iterations = cnt.iters;
  loc.sweeps = sweeps;
  loc.matvecs = cnt.matvecs;
  loc.converged = conv ? 1 : 0;
  loc.rel_residual = worst;
  loc.seconds = std::chrono::duration<double>(t1 - t0).count();
  if (st) *st = loc;
  if (!conv) {
    set_error("solver stopped at its caps: relative residual " + std::to_string(worst));
    return VOXCAP_ERR_NOT_CONVERGED;
  }
  return VOXCAP_OK;
}

// ------------------------------------------------------------------ capacitance
// B[jj][p] = 1 on the conductor panels of conductor j0 + jj, else 0
__global__ void k_unit_rhs(int64_t N, int j0, int nj, const int8_t* kind, const int16_t* owner, double* B) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nj) return;
  const int j = j0 + (int)(t / N);
  const int64_t p = t % N;
  B[t] = (kind[p] == 0 && owner[p] == j) ? 1.0 : 0.0;
}

// C'[s][i][jj] = sum_{p in structure s, conductor i} qscale_p rho_jj[p]
__global__ void k_cap_reduce(int64_t N, int m, int nj, const int64_t* off, const int64_t* ncond,
                             const int16_t* owner, const double* qscale, const double* rho,
                             double* Cn) {
  __shared__ double sh[32];
  const int s = blockIdx.x, i = blockIdx.y, jj = blockIdx.z;
  const int64_t lo = off[s], hi = lo + ncond[s];
  double acc = 0.0;
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x)
    if (owner[p] == i) acc += qscale[p] * rho[(int64_t)jj * N + p];
  double v = block_sum(acc, sh);
  if (threadIdx.x == 0) Cn[((int64_t)s * m + i) * nj + jj] = v;
}

// Columns j0 .. j1-1 of the capacitance matrices (Eq. 8): one unit-potential
// solve per conductor in the range, all in one batch, then the charge sums.
// Every column is solved exactly as in the full batch (its solve does not
// depend on the other columns), so column blocks computed apart -- e.g. on
// different GPUs -- assemble into the same matrix bit for bit.
int capacitance_cols(Handle& h, double tol, int j0, int j1, double* C_host, double* rho_dev, voxcap_stats* st) {
  const int m = h.pan.m_max;
  const int S = h.pan.S;
  const int64_t N = h.pan.N;
  VC_CHECK(m > 0, VOXCAP_ERR_NO_CONDUCTOR, "no conductor in the material table");
  VC_CHECK(j0 >= 0 && j1 > j0 && j1 <= m, VOXCAP_ERR_ARG, "conductor range outside [0, m)");
  const int nj = j1 - j0;
  VC_TRY(h.rhs.alloc((size_t)N * m));
  VC_TRY(h.rho.alloc((size_t)N * m));
  const int TB = 256;
  k_unit_rhs<<<(unsigned)((N * nj + TB - 1) / TB), TB, 0, h.stream>>>(N, j0, nj, h.pan.kind.p, h.pan.owner.p,
                                                                       h.rhs.p); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  int rc = solve(h, h.rhs.p, nj, tol, h.rho.p, st, false);
  if (rc != VOXCAP_OK && rc != VOXCAP_ERR_NOT_CONVERGED) return rc;
  h.have_rho = (j0 == 0 && j1 == m);   // the adjoint gradient needs every column
  DBuf<int64_t> offd, ncd;
  DBuf<double> Cn;
  VC_TRY(offd.alloc(S));
  VC_TRY(ncd.alloc(S));
  VC_TRY(Cn.alloc((size_t)S * m * nj));
  VC_CUDA(cudaMemcpyAsync(offd.p, h.pan.off.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, h.stream));
  VC_CUDA(cudaMemcpyAsync(ncd.p, h.pan.nc.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, h.stream));
  k_cap_reduce<<<dim3(S, m, nj), TB, 0, h.stream>>>(N, m, nj, offd.p, ncd.p, h.pan.owner.p, h.pan.qscale.p,
                                                   h.rho.p, Cn.p); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  std::vector<double> cn((size_t)S * m * nj);
  VC_CUDA(cudaMemcpyAsync(cn.data(), Cn.p, sizeof(double) * cn.size(), cudaMemcpyDeviceToHost, h.stream));
  VC_CUDA(cudaStreamSynchronize(h.stream));
  const double eps0 = 8.8541878128e-12;
  for (size_t q = 0; q < cn.size(); ++q) C_host[q] = eps0 * h.dv * cn[q];
  if (rho_dev)
    VC_CUDA(cudaMemcpy(rho_dev, h.rho.p, sizeof(double) * (size_t)N * nj, cudaMemcpyDeviceToDevice));
  return rc;
}

int capacitance(Handle& h, double tol, double* C_host, double* rho_dev, voxcap_stats* st) {
  VC_CHECK(h.pan.m_max > 0, VOXCAP_ERR_NO_CONDUCTOR, "no conductor in the material table");
  return capacitance_cols(h, tol, 0, h.pan.m_max, C_host, rho_dev, st);
}

}  // namespace vc
