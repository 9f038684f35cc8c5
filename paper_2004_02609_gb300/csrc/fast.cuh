// Compile-time Stockham stages for the products on the common padded
// lengths (2^a * 9 with two or three radix stages): the length, the radices,
// the tile width and the thread count are template parameters, so every
// index of a stage is constant-folded, and a tile needs one shared-memory
// buffer (a middle stage runs in place: each thread holds all of its
// butterflies in registers across a barrier).  Used by the FP32 passes in
// fast_{x,y,z}.cu and by the FP64 y passes; the generic passes in mvm.cu /
// zmac.cuh cover every other length and the FP64 x and z passes.
#pragma once
#include "internal.h"

namespace vc {
namespace fast {

using C = float2;

// A plan of two (R3 == 1) or three radix stages; stage s combines
// sub-transforms of length NS_s with radix R_s (Stockham autosort).
template <int R1_, int R2_, int R3_> struct Plan {
  static constexpr int R1 = R1_, R2 = R2_, R3 = R3_;
  static constexpr int L = R1 * R2 * R3;
  static constexpr int NST = R3 > 1 ? 3 : 2;
  static constexpr int RL = R3 > 1 ? R3 : R2;            // radix of the last stage
  static constexpr int NSL = L / RL;                     // its sub-transform length
};

// The helpers below take the complex type CT (float2, or double2 for the
// FP64 y passes) from their table or buffer pointer.

// v[r] *= w_r (conjugated for the inverse), w_r = tw[k (R-1) + r - 1]
template <int R, bool INV, typename CT>
__device__ __forceinline__ void twiddle(CT* v, const CT* __restrict__ tw, int k) {
  const CT* w = tw + k * (R - 1);
#pragma unroll
  for (int r = 1; r < R; ++r) {
    CT ww = w[r - 1];
    if (INV) ww.y = -ww.y;
    v[r] = cmul(v[r], ww);
  }
}

// One stage (radix R, sub-transform length NS) over TX interleaved lines of
// length L; butterfly item = (j, c) with c = item % TX fastest, spread over
// NT threads.  ld(c, pos) gives the input, st(c, pos, v) takes the output.
// All inputs of a thread's butterflies are loaded before any is transformed,
// so that a stage reading HBM keeps all of its loads in flight at once.
// RIN = R / 2 (first stage only): inputs at positions >= L / 2 are the zero
// padding, neither read nor added.  ROUT < R: only outputs r < ROUT of a
// butterfly are needed (the last stage of a transform whose result is cut to
// fewer than L / 2 positions); the others are not computed.
template <int L, int R, int NS, int TX, int NT, bool INV, int RIN = R, int ROUT = R, typename CT, typename Ld,
          typename St>
__device__ __forceinline__ void stage(const CT* __restrict__ tw, Ld ld, St st) {
  constexpr int NB = L / R, TOT = NB * TX, IT = (TOT + NT - 1) / NT;
  static_assert(RIN == R || (RIN * 2 == R && NS == 1), "half inputs in a first stage only");
  CT v[IT][R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int item = it * NT + (int)threadIdx.x;
    if (TOT % NT == 0 || item < TOT) {
      const int c = item % TX, j = item / TX;
#pragma unroll
      for (int r = 0; r < RIN; ++r) v[it][r] = ld(c, j + r * NB);
    }
  }
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int item = it * NT + (int)threadIdx.x;
    if (TOT % NT == 0 || item < TOT) {
      const int c = item % TX, j = item / TX, k = j % NS;
      if (NS > 1) twiddle<R, INV>(v[it], tw, k);
      dft<R, CT, (RIN < R)>(v[it], INV);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < ROUT; ++r) st(c, base + r * NS, v[it][r]);
    }
  }
}

// The same stage in place on buf (element (pos, c) at pos * PT + c, pitch
// PT >= TX): all inputs of a thread's butterflies are read, the block
// synchronises, the outputs are written, and the block synchronises again.
// ld(c, pos) reads the input (default: buf itself).
template <int L, int R, int NS, int TX, int NT, bool INV, int PT = TX, int RIN = R, int ROUT = R, typename CT,
          typename Ld>
__device__ __forceinline__ void stage_inplace_ld(CT* buf, const CT* __restrict__ tw, Ld ld) {
  constexpr int NB = L / R, TOT = NB * TX, IT = (TOT + NT - 1) / NT;
  static_assert(RIN == R || (RIN * 2 == R && NS == 1), "half inputs in a first stage only");
  CT v[IT][R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int item = it * NT + (int)threadIdx.x;
    if (TOT % NT == 0 || item < TOT) {
      const int c = item % TX, j = item / TX;
#pragma unroll
      for (int r = 0; r < RIN; ++r) v[it][r] = ld(c, j + r * NB);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int item = it * NT + (int)threadIdx.x;
    if (TOT % NT == 0 || item < TOT) {
      const int c = item % TX, j = item / TX, k = j % NS;
      if (NS > 1) twiddle<R, INV>(v[it], tw, k);
      dft<R, CT, (RIN < R)>(v[it], INV);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < ROUT; ++r) buf[(base + r * NS) * PT + c] = v[it][r];
    }
  }
  __syncthreads();
}

template <int L, int R, int NS, int TX, int NT, bool INV, int PT = TX, int RIN = R, int ROUT = R, typename CT>
__device__ __forceinline__ void stage_inplace(CT* buf, const CT* __restrict__ tw) {
  stage_inplace_ld<L, R, NS, TX, NT, INV, PT, RIN, ROUT>(buf, tw,
                                                         [&](int c, int pos) -> CT { return buf[pos * PT + c]; });
}

// cp.async of 8 bytes global -> shared (cached in L1 and L2), its group
// commit, and the wait for all of this thread's groups
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
// one complex value (8 or 16 bytes) global -> shared
template <typename CT>
__device__ __forceinline__ void cp_async_elem(CT* smem, const CT* gmem) {
  if constexpr (sizeof(CT) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
  else
    cp_async8(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// A whole transform of TX interleaved lines held in buf, every stage in
// place (twiddle tables of the plan's stages at tw + off[s]).  HIN: the
// input lines are zero from position L / 2 on (those entries of buf are
// never read); HOUT: only positions < L / 2 of the result are used (the
// last stage leaves the others unwritten).
// transform_inplace_ld: the same with the first stage's inputs from ld(c, pos).
template <typename P, int TX, int NT, bool INV, int PT = TX, bool HIN = false, bool HOUT = false, typename CT,
          typename Ld>
__device__ __forceinline__ void transform_inplace_ld(CT* buf, const CT* __restrict__ tw, int off2, int off3, Ld ld) {
  constexpr int RL = P::NST == 3 ? P::R3 : P::R2;
  constexpr int ROUT = HOUT ? (RL + 1) / 2 : RL;
  stage_inplace_ld<P::L, P::R1, 1, TX, NT, INV, PT, HIN ? P::R1 / 2 : P::R1>(buf, tw, ld);
  if constexpr (P::NST == 3) {
    stage_inplace<P::L, P::R2, P::R1, TX, NT, INV, PT>(buf, tw + off2);
    stage_inplace<P::L, P::R3, P::R1 * P::R2, TX, NT, INV, PT, P::R3, ROUT>(buf, tw + off3);
  } else {
    stage_inplace<P::L, P::R2, P::R1, TX, NT, INV, PT, P::R2, ROUT>(buf, tw + off2);
  }
}

template <typename P, int TX, int NT, bool INV, int PT = TX, bool HIN = false, bool HOUT = false, typename CT>
__device__ __forceinline__ void transform_inplace(CT* buf, const CT* __restrict__ tw, int off2, int off3) {
  transform_inplace_ld<P, TX, NT, INV, PT, HIN, HOUT>(buf, tw, off2, off3,
                                                      [&](int c, int pos) -> CT { return buf[pos * PT + c]; });
}

// copy n complex values to shared memory (caller synchronises)
template <int NT, typename CT>
__device__ __forceinline__ void load_table(CT* dst, const CT* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += NT) dst[i] = src[i];
}

}  // namespace fast

// ---- dispatch (fast_*.cu): each returns VOXCAP_ERR_UNSUPPORTED when no
// compiled plan matches the handle's lengths, so that the caller falls back
// to the generic passes.
bool fast_plan_ok(const Plan1D<float2>& p);
int fast_ypass(const Handle& h, bool inv, int G, const float2* in, float2* out, int64_t in_bstride,
               int64_t out_bstride, int B, int variant, cudaStream_t st);
// the FP64 y passes on the same compiled plans (persistent form), for the
// FP64 products
int fast_ypass_f64(const Handle& h, bool inv, int G, const double2* in, double2* out, int64_t in_bstride,
                   int64_t out_bstride, int B, cudaStream_t st);
bool fast_z_ok(const Handle& h);
int fast_zpass(const Handle& h, float2* data, int B, cudaStream_t st);
// forward x passes (panel scatter + R2C along x; C2R along x + panel gather)
bool fast_x_ok(const Handle& h);
int fast_xfwd(const Handle& h, const float* x, float2* out, int nrhs, cudaStream_t st);
int fast_xinv(const Handle& h, const float2* in, const float* x, float* y, int nrhs, cudaStream_t st);

}  // namespace vc
