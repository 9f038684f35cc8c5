// Shared device/host helpers of the VoxCap GB300 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/voxcap.h"

namespace vc {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
// host-side count of kernel launches issued by the library
void note_launch();
int64_t launch_count();
struct Status {
  int code = VOXCAP_OK;
};

#define VC_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::vc::set_error(std::string("CUDA error at ") + __FILE__ + ":" +       \
                      std::to_string(__LINE__) + ": " +                       \
                      cudaGetErrorString(e_));                                \
      return VOXCAP_ERR_CUDA;                                                 \
    }                                                                         \
  } while (0)

#define VC_CHECK(cond, code, msg)                                             \
  do {                                                                        \
    if (!(cond)) {                                                            \
      ::vc::set_error(msg);                                                   \
      return (code);                                                          \
    }                                                                         \
  } while (0)

#define VC_TRY(expr)                                                          \
  do {                                                                        \
    int rc_ = (expr);                                                         \
    if (rc_ != VOXCAP_OK) return rc_;                                         \
  } while (0)

// ---------------------------------------------------------------- complex
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using C_t = typename cplx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C c; c.x = a; c.y = b; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i : (x + iy)(-i) = y - ix
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return mk<C>(a.y, -a.x); }
// multiply by +i
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { return mk<C>(-a.y, a.x); }

// ---------------------------------------------------------------- FFT plans
constexpr int kMaxStages = 24;

// A 1-D transform of length L factored into radices r[0..nst) in {2,3,4,5,7,8}.
// tw points to L complex twiddles tw[m] = exp(-2 pi i m / L) in device memory.
template <typename C> struct Plan1D {
  int L;
  int nst;
  int radix[kMaxStages];
  const C* tw;
};

bool factor_length(int L, int* radix, int* nst);   // host: false if not 2/3/5/7-smooth

// ---------------------------------------------------------------- Stockham
// Small DFTs: y[k] = sum_j v[j] w^(jk), w = exp(-+ 2 pi i / R).
template <int R, typename C>
__device__ __forceinline__ void dft(C* v, bool inv, const C* __restrict__ tw, int L) {
  if constexpr (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    t3 = inv ? cmul_pi(t3) : cmul_mi(t3);
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
  } else if constexpr (R == 8) {
    // split into even / odd radix-4 halves
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft<4, C>(e, inv, tw, L);
    dft<4, C>(o, inv, tw, L);
    using T = decltype(C::x);
    const T h = (T)0.70710678118654752440084436210484903928;
    // w8^k for k = 1,2,3 (forward: exp(-i pi k / 4))
    C w1 = inv ? mk<C>(h, h) : mk<C>(h, -h);
    C o1 = cmul(o[1], w1);
    C o2 = inv ? cmul_pi(o[2]) : cmul_mi(o[2]);
    C w3 = inv ? mk<C>(-h, h) : mk<C>(-h, -h);
    C o3 = cmul(o[3], w3);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  } else {
    // odd prime radix: direct sum with the roots taken from the length-L table
    C y[R];
    const int step = L / R;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      C acc = v[0];
#pragma unroll
      for (int j = 1; j < R; ++j) {
        C w = tw[((j * k) % R) * step];
        if (inv) w.y = -w.y;
        acc = cadd(acc, cmul(v[j], w));
      }
      y[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = y[k];
  }
}

// One Stockham autosort stage (radix R, Ns = product of the radices done so
// far) over `nlines` interleaved lines: element (pos, line) at pos*ld + line.
template <int R, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst,
                                               int L, int Ns, int nlines, int ld,
                                               const C* __restrict__ tw, bool inv) {
  const int nb = L / R;
  const int twstride = L / (Ns * R);
  for (int t = threadIdx.x; t < nb * nlines; t += blockDim.x) {
    const int line = t % nlines;
    const int j = t / nlines;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * ld + line];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = __ldg(&tw[r * k * twstride]);
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dft<R, C>(v, inv, tw, L);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * ld + line] = v[r];
  }
}

// Transform `nlines` lines held in shared memory (layout pos*ld + line);
// `scr` is a scratch area of the same size.  Returns the buffer that holds
// the result (buf or scr).  All threads of the block must call it.
template <typename C>
__device__ C* fft_lines(C* buf, C* scr, int nlines, int ld, const Plan1D<C>& p, bool inv) {
  C* src = buf;
  C* dst = scr;
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    switch (R) {
      case 2: stockham_stage<2, C>(src, dst, p.L, Ns, nlines, ld, p.tw, inv); break;
      case 3: stockham_stage<3, C>(src, dst, p.L, Ns, nlines, ld, p.tw, inv); break;
      case 4: stockham_stage<4, C>(src, dst, p.L, Ns, nlines, ld, p.tw, inv); break;
      case 5: stockham_stage<5, C>(src, dst, p.L, Ns, nlines, ld, p.tw, inv); break;
      case 7: stockham_stage<7, C>(src, dst, p.L, Ns, nlines, ld, p.tw, inv); break;
      default: stockham_stage<8, C>(src, dst, p.L, Ns, nlines, ld, p.tw, inv); break;
    }
    __syncthreads();
    Ns *= R;
    C* t = src; src = dst; dst = t;
  }
  return src;
}

// ---------------------------------------------------------------- scan
// exclusive prefix sum of n int32 values in place on the device; tmp must hold
// at least scan_tmp_elems(n) ints.
int64_t scan_tmp_elems(int64_t n);
int exclusive_scan_i32(int32_t* data, int64_t n, int32_t* tmp, int64_t* total_host,
                       cudaStream_t st);

}  // namespace vc
