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
void adjust_launch_count(int64_t delta);
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

// Exact x / d for x < 2^16 and 1 <= d < 2^16 by a multiply-high with
// m = ceil(2^32 / d) (the error term x * (m d - 2^32) / 2^32 stays below 1/d).
struct FastDiv {
  uint32_t d, m;
};
__host__ __device__ __forceinline__ FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.m = d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + d - 1) / d);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return f.d <= 1 ? x : __umulhi(x, f.m);
}

// A 1-D transform of length L factored into radices r[0..nst) in {2,3,4,5,7,8,9,16}.
// Stage s combines sub-transforms of length Ns[s] with radix[s]; its twiddles
// exp(-2 pi i r k / (Ns R)), k < Ns, 1 <= r < R, sit at stw[twoff[s] + k (R-1) + r - 1].
template <typename C> struct Plan1D {
  int L;
  int nst;
  int radix[kMaxStages];
  int Ns[kMaxStages];
  FastDiv fNs[kMaxStages];
  int twoff[kMaxStages];
  int twn;            // total number of stage twiddles
  const C* stw;       // stage twiddles, device memory (copied to shared memory by the kernels)
};

bool factor_length(int L, int* radix, int* nst);   // host: false if not 2/3/5/7-smooth
double fft_cost(int L);                           // host: relative cost of one padded length

// Copy the stage twiddles of a plan into shared memory (caller synchronises).
template <typename C> __device__ __forceinline__ void load_twiddles(C* dst, const Plan1D<C>& p) {
  for (int i = threadIdx.x; i < p.twn; i += blockDim.x) dst[i] = p.stw[i];
}

// ---------------------------------------------------------------- butterflies
// y[k] = sum_j v[j] w^(jk), w = exp(-2 pi i / R) (forward) or its conjugate.
template <typename C> __device__ __forceinline__ C cmul_i(C a, bool inv) {   // a * (-i) fwd, a * (+i) inv
  return inv ? cmul_pi(a) : cmul_mi(a);
}

// HIN: only v[0 .. R/2) are given, the upper half of the inputs is zero (a
// zero-padded line's first stage); even R only.
template <int R, typename C, bool HIN = false> __device__ __forceinline__ void dft(C* v, bool inv) {
  using T = decltype(C::x);
  static_assert(!HIN || R == 2 || R == 4 || R == 8 || R == 16, "half-input DFT of an even radix only");
  if constexpr (R == 2 && HIN) {
    v[1] = v[0];
  } else if constexpr (R == 4 && HIN) {
    const C a = v[0], b = v[1], bi = cmul_i(b, inv);
    v[0] = cadd(a, b); v[2] = csub(a, b);
    v[1] = cadd(a, bi); v[3] = csub(a, bi);
  } else if constexpr (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if constexpr (R == 3) {
    const T s = (T)0.8660254037844386467637;
    C a = cadd(v[1], v[2]);
    C t = csub(v[0], cscale(a, (T)0.5));
    C u = cmul_i(cscale(csub(v[1], v[2]), s), inv);
    v[0] = cadd(v[0], a);
    v[1] = cadd(t, u);
    v[2] = csub(t, u);
  } else if constexpr (R == 4) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = cmul_i(csub(v[1], v[3]), inv);
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
  } else if constexpr (R == 5) {
    const T c1 = (T)0.3090169943749474241023, c2 = (T)-0.8090169943749474241023;
    const T s1 = (T)0.9510565162951535721164, s2 = (T)0.5877852522924731291687;
    C a = cadd(v[1], v[4]), b = cadd(v[2], v[3]);
    C d = csub(v[1], v[4]), e = csub(v[2], v[3]);
    C t1 = cadd(v[0], cadd(cscale(a, c1), cscale(b, c2)));
    C t2 = cadd(v[0], cadd(cscale(a, c2), cscale(b, c1)));
    C u1 = cmul_i(cadd(cscale(d, s1), cscale(e, s2)), inv);
    C u2 = cmul_i(csub(cscale(d, s2), cscale(e, s1)), inv);
    v[0] = cadd(v[0], cadd(a, b));
    v[1] = cadd(t1, u1); v[4] = csub(t1, u1);
    v[2] = cadd(t2, u2); v[3] = csub(t2, u2);
  } else if constexpr (R == 7) {
    const T c1 = (T)0.623489801858733530525, c2 = (T)-0.2225209339563144042889,
            c3 = (T)-0.9009688679024191262361;
    const T s1 = (T)0.7818314824680298087084, s2 = (T)0.9749279121818236070181,
            s3 = (T)0.4338837391175581204758;
    C a1 = cadd(v[1], v[6]), a2 = cadd(v[2], v[5]), a3 = cadd(v[3], v[4]);
    C d1 = csub(v[1], v[6]), d2 = csub(v[2], v[5]), d3 = csub(v[3], v[4]);
    // cos(2 pi j k / 7) and sin(...) for k = 1, 2, 3 over the pairs j = 1, 2, 3
    C t1 = cadd(v[0], cadd(cscale(a1, c1), cadd(cscale(a2, c2), cscale(a3, c3))));
    C t2 = cadd(v[0], cadd(cscale(a1, c2), cadd(cscale(a2, c3), cscale(a3, c1))));
    C t3 = cadd(v[0], cadd(cscale(a1, c3), cadd(cscale(a2, c1), cscale(a3, c2))));
    C u1 = cmul_i(cadd(cscale(d1, s1), cadd(cscale(d2, s2), cscale(d3, s3))), inv);
    C u2 = cmul_i(csub(cscale(d1, s2), cadd(cscale(d2, s3), cscale(d3, s1))), inv);
    C u3 = cmul_i(cadd(cscale(d1, s3), csub(cscale(d3, s2), cscale(d2, s1))), inv);
    v[0] = cadd(v[0], cadd(a1, cadd(a2, a3)));
    v[1] = cadd(t1, u1); v[6] = csub(t1, u1);
    v[2] = cadd(t2, u2); v[5] = csub(t2, u2);
    v[3] = cadd(t3, u3); v[4] = csub(t3, u3);
  } else if constexpr (R == 9 || R == 16) {
    // R = Q * Q (Q = 3 or 4): X[q + Q p] = sum_k1 wQ^(k1 p) [ wR^(k1 q) sum_n2 x[k1 + Q n2] wQ^(n2 q) ]
    constexpr int Q = R == 9 ? 3 : 4;
    C a[Q][Q];
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) a[k1][n2] = (HIN && n2 >= Q / 2) ? mk<C>(0, 0) : v[k1 + Q * n2];
      dft<Q, C, HIN>(a[k1], inv);
    }
#pragma unroll
    for (int k1 = 1; k1 < Q; ++k1)
#pragma unroll
      for (int q = 1; q < Q; ++q) {
        const int mm = k1 * q;                     // exponent of wR
        T wr, wi;
        if constexpr (R == 16) {
          wr = mm == 1 ? (T)0.9238795325112867561282 : mm == 2 ? (T)0.7071067811865475244008
             : mm == 3 ? (T)0.3826834323650897717285 : mm == 4 ? (T)0.0
             : mm == 6 ? (T)-0.7071067811865475244008 : (T)-0.9238795325112867561282;
          wi = mm == 1 ? (T)-0.3826834323650897717285 : mm == 2 ? (T)-0.7071067811865475244008
             : mm == 3 ? (T)-0.9238795325112867561282 : mm == 4 ? (T)-1.0
             : mm == 6 ? (T)-0.7071067811865475244008 : (T)0.3826834323650897717285;
        } else {
          wr = mm == 1 ? (T)0.7660444431189780352024 : mm == 2 ? (T)0.1736481776669303488517
                                                     : (T)-0.9396926207859083840541;
          wi = mm == 1 ? (T)-0.6427876096865393263226 : mm == 2 ? (T)-0.9848077530122080593667
                                                     : (T)-0.3420201433256687330441;
        }
        if (inv) wi = -wi;
        a[k1][q] = cmul(a[k1][q], mk<C>(wr, wi));
      }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      C b[Q];
#pragma unroll
      for (int k1 = 0; k1 < Q; ++k1) b[k1] = a[k1][q];
      dft<Q, C>(b, inv);
#pragma unroll
      for (int p = 0; p < Q; ++p) v[q + Q * p] = b[p];
    }
  } else {   // R == 8: two radix-4 halves
    using TT = T;
    C e[4] = {v[0], v[2], HIN ? mk<C>(0, 0) : v[4], HIN ? mk<C>(0, 0) : v[6]};
    C o[4] = {v[1], v[3], HIN ? mk<C>(0, 0) : v[5], HIN ? mk<C>(0, 0) : v[7]};
    dft<4, C, HIN>(e, inv);
    dft<4, C, HIN>(o, inv);
    const TT h = (TT)0.70710678118654752440084436210484903928;
    C w1 = inv ? mk<C>(h, h) : mk<C>(h, -h);
    C o1 = cmul(o[1], w1);
    C o2 = cmul_i(o[2], inv);
    C w3 = inv ? mk<C>(-h, h) : mk<C>(-h, -h);
    C o3 = cmul(o[3], w3);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
}

// One Stockham autosort stage over NL interleaved lines (element (pos, line)
// at pos*ld + line); tw = this stage's twiddles in shared memory.
template <int R, int NL, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst, int L,
                                               int Ns, const FastDiv& fNs, int ld,
                                               const C* __restrict__ tw, bool inv) {
  const int nb = L / R;
  const int total = nb * NL;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int j = t / NL;
    const int line = t - j * NL;
    const int k = j - (int)fdiv((uint32_t)j, fNs) * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * ld + line];
    if (Ns > 1) {
      const C* w = tw + k * (R - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C ww = w[r - 1];
        if (inv) ww.y = -ww.y;
        v[r] = cmul(v[r], ww);
      }
    }
    dft<R, C>(v, inv);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * ld + line] = v[r];
  }
}

// Transform NL lines held in shared memory (layout pos*ld + line); `scr` is a
// scratch area of the same size and `stw` the plan's stage twiddles in shared
// memory.  Returns the buffer holding the result.  All threads of the block
// must call it.
template <int NL, typename C>
__device__ C* fft_lines(C* buf, C* scr, int ld, const Plan1D<C>& p, const C* stw, bool inv) {
  C* src = buf;
  C* dst = scr;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    const C* tw = stw + p.twoff[s];
    switch (R) {
      case 2: stockham_stage<2, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      case 3: stockham_stage<3, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      case 4: stockham_stage<4, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      case 5: stockham_stage<5, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      case 7: stockham_stage<7, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      case 9: stockham_stage<9, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      case 16: stockham_stage<16, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
      default: stockham_stage<8, NL, C>(src, dst, p.L, p.Ns[s], p.fNs[s], ld, tw, inv); break;
    }
    __syncthreads();
    C* t = src; src = dst; dst = t;
  }
  return src;
}

// One Stockham stage over `nlines` lines whose inputs come from ld(line, pos)
// and whose outputs go to st(line, pos, value), so that a pass can read its
// first stage straight from global memory and write its last stage straight
// back.  Requires nb * nlines < 2^16 (nb = L / R).
template <int R, typename C, typename Ld, typename St>
__device__ __forceinline__ void stockham_stage_io(int L, int Ns, const FastDiv& fNs, int nlines,
                                                  const FastDiv& fnl, const C* __restrict__ tw,
                                                  bool inv, Ld ld, St st) {
  const int nb = L / R;
  const int total = nb * nlines;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int j = (int)fdiv((uint32_t)t, fnl);
    const int line = t - j * nlines;
    const int k = j - (int)fdiv((uint32_t)j, fNs) * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(line, j + r * nb);
    if (Ns > 1) {
      const C* w = tw + k * (R - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C ww = w[r - 1];
        if (inv) ww.y = -ww.y;
        v[r] = cmul(v[r], ww);
      }
    }
    dft<R, C>(v, inv);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st(line, base + r * Ns, v[r]);
  }
}

// Stage s of plan p through stockham_stage_io (stw: the plan's stage twiddles).
template <typename C, typename Ld, typename St>
__device__ __forceinline__ void stage_io(const Plan1D<C>& p, int s, const C* stw, int nlines,
                                         const FastDiv& fnl, bool inv, Ld ld, St st) {
  const C* tw = stw + p.twoff[s];
  switch (p.radix[s]) {
    case 2: stockham_stage_io<2, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    case 3: stockham_stage_io<3, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    case 4: stockham_stage_io<4, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    case 5: stockham_stage_io<5, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    case 7: stockham_stage_io<7, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    case 9: stockham_stage_io<9, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    case 16: stockham_stage_io<16, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
    default: stockham_stage_io<8, C>(p.L, p.Ns[s], p.fNs[s], nlines, fnl, tw, inv, ld, st); break;
  }
}

// Dispatch a power-of-two tile width (1..16) to a template instantiation.
#define VC_TILE_DISPATCH(W, F) \
  switch (W) {                 \
    case 1: F(1); break;       \
    case 2: F(2); break;       \
    case 4: F(4); break;       \
    case 8: F(8); break;       \
    default: F(16); break;     \
  }

// ---------------------------------------------------------------- scan
// exclusive prefix sum of n int32 values in place on the device; tmp must hold
// at least scan_tmp_elems(n) ints.
int64_t scan_tmp_elems(int64_t n);
int exclusive_scan_i32(int32_t* data, int64_t n, int32_t* tmp, int64_t* total_host,
                       cudaStream_t st);

}  // namespace vc
