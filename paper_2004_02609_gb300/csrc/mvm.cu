// FFT-accelerated products with the system matrix (Eqs. 9-11) and its
// transpose, in FP32 or FP64.
//
// Forward (y = A x): the charges of the panels of each orientation b are
// scattered onto the b-face grid (zero elsewhere, never materialised beyond
// one row), transformed along x, y, z to the padded size M (R2C along x),
// multiplied by the 15 kernel spectra (6 potential + 9 field blocks, Eq. 12
// folds the other three potential blocks), transformed back, and gathered:
// a conductor row takes the potential C^a at its face, a dielectric row
// takes I' x + D^a (Eqs. 4, 9-11).
//
// Passes (one kernel each):
//   xfwd  gather panel values into face rows, R2C along x (two real rows per
//         complex line), half-voxel phase on the x grid
//   yfwd  C2C along y (zero-padded input), phase on the y grid
//   zmac  C2C along z, phase on the z grid, spectral multiply-accumulate,
//         output phase on z outputs, inverse along z, truncation to N+1 planes
//   yinv  inverse along y (truncated to N+1 rows), output phase on y outputs
//   xinv  output phase on x outputs, C2R along x (two real rows per line),
//         gather at the panels
// The transposed product runs the same passes with the panel values split
// by row kind (6 input grids), the conjugated kernels and 3 output grids.
// The generic z pass lives in zmac.cuh (one translation unit per precision
// and direction).  FP32 products on the compiled lengths run the passes of
// fast_{x,y,z}.cu instead (path 1 and its launch variants, tuned at set-up
// against the generic passes' radix orders and tile widths); FP64 products
// run the compiled y passes there and the generic x and z passes.
#include <type_traits>

#include "fast.cuh"
#include "internal.h"

namespace vc {

struct MvmArgs {
  Geom g;
  int nrhs;
  int64_t N;
  const int32_t* fmap;
  const int8_t* kind;
  const double* idiag;
  const float* idiag_f;
};

template <typename T> __device__ __forceinline__ T idiag_of(const MvmArgs& a, int64_t p);
template <> __device__ __forceinline__ float idiag_of<float>(const MvmArgs& a, int64_t p) { return a.idiag_f[p]; }
template <> __device__ __forceinline__ double idiag_of<double>(const MvmArgs& a, int64_t p) { return a.idiag[p]; }

// ------------------------------------------------------------------ xfwd
// Forward: line l = rows (2l, 2l+1) of grid g.  Adjoint: line l = row l of
// the conductor-source grid g (real part) and dielectric-source grid g (imag).
template <typename T, bool ADJ, int NL>
__global__ void k_xfwd(MvmArgs a, const T* __restrict__ xin, C_t<T>* __restrict__ out,
                       Plan1D<C_t<T>> plan, const C_t<T>* __restrict__ phx) {
  using C = C_t<T>;
  extern __shared__ unsigned char smem_raw[];
  const Geom& g = a.g;
  const int M = g.Mx, H = g.Hx;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* scr = buf + (size_t)M * NL;
  C* stw = scr + (size_t)M * NL;
  load_twiddles(stw, plan);
  const int z = blockIdx.y;
  const int bg = blockIdx.z;             // b * 3 + grid
  const int grid = bg % 3, b = bg / 3;
  const int s = b / a.nrhs, r = b % a.nrhs;
  const int nlines_total = ADJ ? g.Ly : (g.Ly + 1) / 2;
  const int l0 = blockIdx.x * NL;
  const int32_t* fm = a.fmap + (((int64_t)s * 3 + grid) * g.Lz + z) * ((int64_t)g.Ly * g.Lx);
  const T* xr = xin + (int64_t)r * a.N;
  for (int t = threadIdx.x; t < M * NL; t += blockDim.x) {
    const int l = t % NL, x = t / NL;
    T re = 0, im = 0;
    const int line = l0 + l;
    if (x < g.Lx && line < nlines_total) {
      if (!ADJ) {
        const int y0 = 2 * line, y1 = y0 + 1;
        int p0 = fm[(int64_t)y0 * g.Lx + x];
        if (p0 >= 0) re = xr[p0];
        if (y1 < g.Ly) {
          int p1 = fm[(int64_t)y1 * g.Lx + x];
          if (p1 >= 0) im = xr[p1];
        }
      } else {
        int p = fm[(int64_t)line * g.Lx + x];
        if (p >= 0) {
          if (a.kind[p] == 0) re = xr[p]; else im = xr[p];
        }
      }
    }
    buf[x * NL + l] = mk<C>(re, im);
  }
  __syncthreads();
  C* res = fft_lines<NL>(buf, scr, NL, plan, stw, false);
  const int GI = ADJ ? 6 : 3;
  for (int t = threadIdx.x; t < H * NL; t += blockDim.x) {
    const int l = t % NL, k = t / NL;
    const int line = l0 + l;
    if (line >= nlines_total) continue;
    C zk = res[k * NL + l];
    C zc = cconj(res[((M - k) % M) * NL + l]);
    C A = cscale(cadd(zk, zc), (T)0.5);
    C B = cscale(cmul_mi(csub(zk, zc)), (T)0.5);
    if (grid == 0) { C ph = phx[k]; A = cmul(A, ph); B = cmul(B, ph); }
    if (!ADJ) {
      const int y0 = 2 * line, y1 = y0 + 1;
      C* o = out + (((int64_t)b * GI + grid) * g.Lz + z) * ((int64_t)g.Ly * H);
      o[(int64_t)y0 * H + k] = A;
      if (y1 < g.Ly) o[(int64_t)y1 * H + k] = B;
    } else {
      C* oc = out + (((int64_t)b * GI + grid) * g.Lz + z) * ((int64_t)g.Ly * H);
      C* od = out + (((int64_t)b * GI + 3 + grid) * g.Lz + z) * ((int64_t)g.Ly * H);
      oc[(int64_t)line * H + k] = A;
      od[(int64_t)line * H + k] = B;
    }
  }
}

// ------------------------------------------------------------------ yfwd / yinv
// in: [B][G][Lz][Lin][H] -> out: [B][G][Lz][Lout][H], transform along the
// second-fastest axis.  Forward: Lin = Ly (zero-padded to My), Lout = My,
// phase after.  Inverse: Lin = My, Lout = Ly (truncated), conj phase before.
// The first stage reads global memory and the last one writes it; shared
// memory holds the lines between stages (a second buffer only when there
// are middle stages).
template <typename T, bool INV, int TX>
__global__ void k_ypass(Geom g, int G, const C_t<T>* __restrict__ in, C_t<T>* __restrict__ out,
                        int64_t in_bstride, int64_t out_bstride,
                        Plan1D<C_t<T>> plan, const C_t<T>* __restrict__ phy) {
  using C = C_t<T>;
  extern __shared__ unsigned char smem_raw[];
  const int M = g.My, H = g.Hx;
  const int nst = plan.nst;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* alt = buf + (size_t)M * TX;
  C* stw = alt + (nst >= 3 ? (size_t)M * TX : 0);
  load_twiddles(stw, plan);
  const int k0 = blockIdx.x * TX;
  const int z = blockIdx.y;
  const int bg = blockIdx.z;           // b * G + grid
  const int grid = bg % G, b = bg / G;
  const bool phase = (grid % 3) == 1;
  const int Lin = INV ? M : g.Ly;
  const int Lout = INV ? g.Ly : M;
  const int ncol = min(TX, H - k0);
  const C* src = in + (int64_t)b * in_bstride + ((int64_t)grid * g.Lz + z) * ((int64_t)Lin * H) + k0;
  C* dst = out + (int64_t)b * out_bstride + ((int64_t)grid * g.Lz + z) * ((int64_t)Lout * H) + k0;
  const FastDiv fTX = make_fastdiv((uint32_t)TX);
  auto gload = [&](int c, int y) -> C {
    C v = mk<C>((T)0, (T)0);
    if (c < ncol && y < Lin) {
      v = src[(int64_t)y * H + c];
      if (INV && phase) v = cmul(v, cconj(phy[y]));
    }
    return v;
  };
  auto gstore = [&](int c, int y, C v) {
    if (c < ncol && y < Lout) {
      if (!INV && phase) v = cmul(v, phy[y]);
      dst[(int64_t)y * H + c] = v;
    }
  };
  __syncthreads();
  if (nst == 1) {
    stage_io(plan, 0, stw, TX, fTX, INV, gload, gstore);
    return;
  }
  stage_io(plan, 0, stw, TX, fTX, INV, gload, [&](int c, int y, C v) { buf[y * TX + c] = v; });
  __syncthreads();
  C* a = buf;
  C* o = alt;
  for (int s = 1; s < nst - 1; ++s) {
    stage_io(plan, s, stw, TX, fTX, INV, [&](int c, int y) { return a[y * TX + c]; },
             [&](int c, int y, C v) { o[y * TX + c] = v; });
    __syncthreads();
    C* t = a; a = o; o = t;
  }
  stage_io(plan, nst - 1, stw, TX, fTX, INV, [&](int c, int y) { return a[y * TX + c]; }, gstore);
}

// ------------------------------------------------------------------ xinv
// Forward: line = row y of output orientation a: potential row (grid a) and
// field row (grid 3+a) -> gather.  Adjoint: line = rows (2l, 2l+1) of grid a.
template <typename T, bool ADJ, int NL>
__global__ void k_xinv(MvmArgs a, const C_t<T>* __restrict__ in, const T* __restrict__ xin,
                       T* __restrict__ yout, T* __restrict__ field, Plan1D<C_t<T>> plan,
                       const C_t<T>* __restrict__ phx) {
  using C = C_t<T>;
  extern __shared__ unsigned char smem_raw[];
  const Geom& g = a.g;
  const int M = g.Mx, H = g.Hx;
  constexpr int GO = ADJ ? 3 : 6;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* scr = buf + (size_t)M * NL;
  C* stw = scr + (size_t)M * NL;
  load_twiddles(stw, plan);
  const int z = blockIdx.y;
  const int bo = blockIdx.z;            // b * 3 + orientation
  const int al = bo % 3, b = bo / 3;
  const int s = b / a.nrhs, r = b % a.nrhs;
  const int nlines_total = ADJ ? (g.Ly + 1) / 2 : g.Ly;
  const int l0 = blockIdx.x * NL;
  const int64_t plane = (int64_t)g.Ly * H;
  const C* srcA;
  const C* srcB;
  if (!ADJ) {
    srcA = in + (((int64_t)b * GO + al) * g.Lz + z) * plane;
    srcB = in + (((int64_t)b * GO + 3 + al) * g.Lz + z) * plane;
  } else {
    srcA = in + (((int64_t)b * GO + al) * g.Lz + z) * plane;
    srcB = srcA;
  }
  for (int t = threadIdx.x; t < M * NL; t += blockDim.x) {
    const int l = t % NL, k = t / NL;
    const int line = l0 + l;
    C v = mk<C>((T)0, (T)0);
    if (line < nlines_total) {
      const int kk = k <= M / 2 ? k : M - k;
      int64_t ra, rb;
      bool hasb = true;
      if (!ADJ) { ra = (int64_t)line * H; rb = ra; }
      else {
        ra = (int64_t)(2 * line) * H;
        rb = ra + H;
        hasb = (2 * line + 1) < g.Ly;
      }
      C A = srcA[ra + kk];
      C B = hasb ? srcB[rb + kk] : mk<C>((T)0, (T)0);
      if (al == 0) { C ph = cconj(phx[kk]); A = cmul(A, ph); B = cmul(B, ph); }
      if (k > M / 2) { A = cconj(A); B = cconj(B); }
      v = cadd(A, cmul_pi(B));
    }
    buf[k * NL + l] = v;
  }
  __syncthreads();
  C* res = fft_lines<NL>(buf, scr, NL, plan, stw, true);
  const int32_t* fm = a.fmap + (((int64_t)s * 3 + al) * g.Lz + z) * ((int64_t)g.Ly * g.Lx);
  const T* xr = xin + (int64_t)r * a.N;
  T* yr = yout + (int64_t)r * a.N;
  for (int t = threadIdx.x; t < g.Lx * NL; t += blockDim.x) {
    const int l = t % NL, x = t / NL;
    const int line = l0 + l;
    if (line >= nlines_total) continue;
    C v = res[x * NL + l];
    if (!ADJ) {
      const int y = line;
      int p = fm[(int64_t)y * g.Lx + x];
      if (p >= 0) {
        if (a.kind[p] == 0) yr[p] = v.x;
        else yr[p] = idiag_of<T>(a, p) * xr[p] + v.y;
      }
      if (field)
        field[(((int64_t)b * 3 + al) * g.Lz + z) * ((int64_t)g.Ly * g.Lx) + (int64_t)y * g.Lx + x] = v.y;
    } else {
      for (int h2 = 0; h2 < 2; ++h2) {
        const int y = 2 * line + h2;
        if (y >= g.Ly) break;
        const T val = h2 == 0 ? v.x : v.y;
        int p = fm[(int64_t)y * g.Lx + x];
        if (p >= 0) yr[p] = val + (a.kind[p] == 1 ? idiag_of<T>(a, p) * xr[p] : (T)0);
        if (field)
          field[(((int64_t)b * 3 + al) * g.Lz + z) * ((int64_t)g.Ly * g.Lx) + (int64_t)y * g.Lx + x] = val;
      }
    }
  }
}

// ------------------------------------------------------------------ driver
template <typename T> static int smem_lines(int L, int cols_per_line, int maxl) {
  const size_t budget = 100 * 1024;
  int nl = (int)(budget / (2 * (size_t)L * cols_per_line * sizeof(C_t<T>)));
  int p = 1;
  while (p * 2 <= nl && p * 2 <= maxl) p *= 2;
  return p;
}

template <typename T>
int mvm(Handle& h, const T* x, T* y, int nrhs, bool adjoint, T* field_out, void* workspace) {
  using C = C_t<T>;
  const Geom& g = h.g;
  const int B = h.pan.S * nrhs;
  const int64_t gX = (int64_t)g.Lz * g.Ly * g.Hx;     // one grid, x-pass layout
  const int64_t gY = (int64_t)g.Lz * g.My * g.Hx;     // one grid, y/z-pass layout
  const size_t need = sizeof(C) * ((size_t)B * 6 * gX + (size_t)B * 6 * gY);
  if (!workspace) {
    VC_TRY(h.ws.alloc(need));
    workspace = h.ws.p;
  }
  C* bufX = reinterpret_cast<C*>(workspace);
  C* bufY = bufX + (size_t)B * 6 * gX;
  MvmArgs a;
  a.g = g;
  a.nrhs = nrhs;
  a.N = h.pan.N;
  a.fmap = h.pan.fmap.p;
  a.kind = h.pan.kind.p;
  a.idiag = h.pan.idiag.p;
  a.idiag_f = h.pan.idiag_f.p;
  const int GI = adjoint ? 6 : 3, GO = adjoint ? 3 : 6;
  const int TB = 256;
  cudaStream_t st = h.stream;
  // compiled-plan passes for FP32 where the lengths allow (path 1); the x
  // passes of the transposed product and of the face-field output stay generic
  const bool fast_x = std::is_same<T, float>::value && h.path == 1 && !adjoint && !field_out && fast_x_ok(h);
  // xfwd
  if (fast_x) {
    VC_TRY(fast_xfwd(h, reinterpret_cast<const float*>(x), reinterpret_cast<float2*>(bufX), nrhs, st));
  } else {
    const int NL = smem_lines<T>(g.Mx, 1, 16);
    const int lines = adjoint ? g.Ly : (g.Ly + 1) / 2;
    dim3 grid((lines + NL - 1) / NL, g.Lz, B * 3);
    size_t sm = (2 * (size_t)g.Mx * NL + plan_of<T>(h, 0).twn) * sizeof(C);
#define VC_XFWD(W)                                                                            \
  if (adjoint) {                                                                              \
    VC_TRY(set_smem(k_xfwd<T, true, W>, sm));                                              \
    k_xfwd<T, true, W><<<grid, TB, sm, st>>>(a, x, bufX, plan_of<T>(h, 0), phase_of<T>(h, 0)); \
  } else {                                                                                    \
    VC_TRY(set_smem(k_xfwd<T, false, W>, sm));                                             \
    k_xfwd<T, false, W><<<grid, TB, sm, st>>>(a, x, bufX, plan_of<T>(h, 0), phase_of<T>(h, 0)); \
  }
    VC_TILE_DISPATCH(NL, VC_XFWD)
#undef VC_XFWD
    ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  const bool fast_y = std::is_same<T, float>::value && h.path == 1 && fast_plan_ok(h.pf[1]);
  // FP64 products: the persistent compiled y passes wherever the plan has one
  // (the generic FP64 passes fit only 2 lines of the longest plans in a CTA)
  const bool fast_y64 = std::is_same<T, double>::value && fast_plan_ok(h.pf[1]);
  const bool fast_z = std::is_same<T, float>::value && h.path == 1 && !adjoint && fast_z_ok(h);
  // yfwd: bufX [B][GI] -> bufY [B][6] (first GI grids)
  // y tiles: the tuned widths for FP32 (4..16 columns), else the widest that fits
  const int TXdef = smem_lines<T>(g.My, 1, 16);
  const int TXf = (sizeof(T) == 4 && h.ytx[0] >= 0) ? (1 << h.ytx[0]) : TXdef;
  const int TXi = (sizeof(T) == 4 && h.ytx[1] >= 0) ? (1 << h.ytx[1]) : TXdef;
  const int ybufs = plan_of<T>(h, 1).nst >= 3 ? 2 : 1;
  if (fast_y) {
    VC_TRY(fast_ypass(h, false, GI, reinterpret_cast<const float2*>(bufX), reinterpret_cast<float2*>(bufY),
                      (int64_t)GI * gX, (int64_t)6 * gY, B, h.yvar[0], st));
  } else if (fast_y64) {
    VC_TRY(fast_ypass_f64(h, false, GI, reinterpret_cast<const double2*>(bufX), reinterpret_cast<double2*>(bufY),
                          (int64_t)GI * gX, (int64_t)6 * gY, B, st));
  } else {
    const int TXy = TXf;
    const int TBy = TXy >= 16 ? 256 : 128;
    size_t sm = (ybufs * (size_t)g.My * TXy + plan_of<T>(h, 1).twn) * sizeof(C);
    dim3 grid((g.Hx + TXy - 1) / TXy, g.Lz, B * GI);
#define VC_YFWD(W)                                                                          \
  VC_TRY(set_smem(k_ypass<T, false, W>, sm));                                            \
  k_ypass<T, false, W><<<grid, TBy, sm, st>>>(g, GI, bufX, bufY, (int64_t)GI * gX, (int64_t)6 * gY, \
                                              plan_of<T>(h, 1), phase_of<T>(h, 1));
    VC_TILE_DISPATCH(TXy, VC_YFWD)
#undef VC_YFWD
    ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  // zmac
  if (fast_z) VC_TRY(fast_zpass(h, reinterpret_cast<float2*>(bufY), B, st));
  else if (adjoint) VC_TRY((zmac_launch<T, true>(h, bufY, B, st)));
  else VC_TRY((zmac_launch<T, false>(h, bufY, B, st)));
  // yinv: bufY [B][6] (first GO grids) -> bufX [B][GO]
  if (fast_y) {
    VC_TRY(fast_ypass(h, true, GO, reinterpret_cast<const float2*>(bufY), reinterpret_cast<float2*>(bufX),
                      (int64_t)6 * gY, (int64_t)GO * gX, B, h.yvar[1], st));
  } else if (fast_y64) {
    VC_TRY(fast_ypass_f64(h, true, GO, reinterpret_cast<const double2*>(bufY), reinterpret_cast<double2*>(bufX),
                          (int64_t)6 * gY, (int64_t)GO * gX, B, st));
  } else {
    const int TXy = TXi;
    const int TBy = TXy >= 16 ? 256 : 128;
    size_t sm = (ybufs * (size_t)g.My * TXy + plan_of<T>(h, 1).twn) * sizeof(C);
    dim3 grid((g.Hx + TXy - 1) / TXy, g.Lz, B * GO);
#define VC_YINV(W)                                                                         \
  VC_TRY(set_smem(k_ypass<T, true, W>, sm));                                            \
  k_ypass<T, true, W><<<grid, TBy, sm, st>>>(g, GO, bufY, bufX, (int64_t)6 * gY, (int64_t)GO * gX, \
                                             plan_of<T>(h, 1), phase_of<T>(h, 1));
    VC_TILE_DISPATCH(TXy, VC_YINV)
#undef VC_YINV
    ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  // xinv + gather
  if (fast_x) {
    VC_TRY(fast_xinv(h, reinterpret_cast<const float2*>(bufX), reinterpret_cast<const float*>(x),
                     reinterpret_cast<float*>(y), nrhs, st));
  } else {
    const int NL = smem_lines<T>(g.Mx, 1, 16);
    const int lines = adjoint ? (g.Ly + 1) / 2 : g.Ly;
    dim3 grid((lines + NL - 1) / NL, g.Lz, B * 3);
    size_t sm = (2 * (size_t)g.Mx * NL + plan_of<T>(h, 0).twn) * sizeof(C);
#define VC_XINV(W)                                                                             \
  if (adjoint) {                                                                               \
    VC_TRY(set_smem(k_xinv<T, true, W>, sm));                                               \
    k_xinv<T, true, W><<<grid, TB, sm, st>>>(a, bufX, x, y, field_out, plan_of<T>(h, 0), phase_of<T>(h, 0)); \
  } else {                                                                                     \
    VC_TRY(set_smem(k_xinv<T, false, W>, sm));                                              \
    k_xinv<T, false, W><<<grid, TB, sm, st>>>(a, bufX, x, y, field_out, plan_of<T>(h, 0), phase_of<T>(h, 0)); \
  }
    VC_TILE_DISPATCH(NL, VC_XINV)
#undef VC_XINV
    ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  return VOXCAP_OK;
}

template int mvm<float>(Handle&, const float*, float*, int, bool, float*, void*);
template int mvm<double>(Handle&, const double*, double*, int, bool, double*, void*);

int mvm_prepare(Handle& h, int nrhs, size_t complex_bytes) {
  return h.ws.alloc(mvm_workspace_bytes(h, nrhs, complex_bytes));
}

// bytes of scratch one product over nrhs columns needs (x-pass and y/z-pass
// intermediates of every batch item)
size_t mvm_workspace_bytes(const Handle& h, int nrhs, size_t complex_bytes) {
  const Geom& g = h.g;
  const size_t B = (size_t)h.pan.S * nrhs;
  const size_t gX = (size_t)g.Lz * g.Ly * g.Hx;
  const size_t gY = (size_t)g.Lz * g.My * g.Hx;
  return complex_bytes * (B * 6 * gX + B * 6 * gY);
}

}  // namespace vc
