// x passes of the forward FP32 product (Eqs. 9-11) on compiled plans.
//
// xfwd: the panel charges of the tile's face rows are scattered straight
// from the panel list (the rows are consecutive in the canonical order, so
// their conductor panels are one contiguous run and their dielectric panels
// another) onto zeroed lines in shared memory -- two real rows per complex
// line --, the line is
// transformed along x, and the half spectra of the two rows are split out,
// given the half-voxel phase of the x grid and written to HBM (row-
// contiguous, coalesced).
// xinv: the potential and field half spectra of the tile's output rows are
// copied into shared memory by cp.async (contiguous runs, all in flight at
// once), extended to the full Hermitian line as potential + i field by the
// first stage as it reads them, transformed back, and gathered at the row's
// panels: a conductor row takes the potential, a dielectric row I' x + the
// field (Eq. 4).
// NL lines share one shared-memory buffer with a pitch of NL + 1 complex
// values, so that reads along x by consecutive lanes avoid bank conflicts.
// The padded length is at least twice the row length: the forward transform
// reads only the lower half of its first stage's inputs, and the inverse
// one computes only the outputs below L / 2.
#include "fast.cuh"

namespace vc {

namespace {

using fast::C;

struct XArgs {
  Geom g;
  int nrhs;
  int64_t N;
  const int32_t* rstart;
  const int32_t* px;
  const float* idiag;
  int64_t R;             // face rows per (structure, kind): 3 Lz Ly
};

template <int R1, int R2, int R3, int NL, int NT>
__global__ void __launch_bounds__(NT) k_xfwd_fast(XArgs a, const float* __restrict__ x, C* __restrict__ out,
                                                  const C* __restrict__ stw, int twn, int off2, int off3,
                                                  const C* __restrict__ phx) {
  using P = fast::Plan<R1, R2, R3>;
  constexpr int L = P::L, H = L / 2 + 1, PT = NL + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tws = buf + L * PT;
  C* phs = tws + twn;                 // half-voxel phases of the x grid
  fast::load_table<NT>(tws, stw, twn);
  fast::load_table<NT>(phs, phx, H);
  const Geom& g = a.g;
  const int z = blockIdx.y;
  const int bg = blockIdx.z;                 // b * 3 + grid
  const int grid = bg % 3, b = bg / 3;
  const int s = b / a.nrhs, r = b % a.nrhs;
  const int nlines = (g.Ly + 1) / 2;         // two rows per complex line
  const int l0 = blockIdx.x * NL;
  const float* xr = x + (int64_t)r * a.N;
  // the tile's rows y0 .. y0 + nrows - 1 are consecutive in the canonical
  // order, so their panels of each kind are one contiguous range; the row
  // starts go to shared memory first
  __shared__ int rs[2][2 * NL + 1];
  const int y0 = 2 * l0;
  const int nrows = min(2 * NL, g.Ly - y0);
  const int64_t row0 = ((int64_t)grid * g.Lz + z) * g.Ly + y0;
  for (int i = threadIdx.x; i < 2 * (nrows + 1); i += NT) {
    const int kind = i / (nrows + 1), k = i - kind * (nrows + 1);
    rs[kind][k] = a.rstart[(2 * (int64_t)s + kind) * a.R + row0 + k];
  }
  for (int i = threadIdx.x; i < (L / 2) * PT; i += NT) buf[i] = mk<C>(0.f, 0.f);   // the upper half is never read
  __syncthreads();
  // scatter: threads over the tile's panels of each kind (independent,
  // coalesced loads); a panel's row by bisection of the row starts
  float* fb = reinterpret_cast<float*>(buf);
#pragma unroll
  for (int kind = 0; kind < 2; ++kind) {
    const int* rk = rs[kind];
    for (int p = rk[0] + threadIdx.x; p < rk[nrows]; p += NT) {
      int lo = 0, hi = nrows;                   // rk[lo] <= p < rk[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rk[mid] <= p) lo = mid;
        else hi = mid;
      }
      fb[2 * (a.px[p] * PT + (lo >> 1)) + (lo & 1)] = xr[p];
    }
  }
  __syncthreads();
  fast::transform_inplace<P, NL, NT, false, PT, true, false>(buf, tws, off2, off3);
  // split the two rows' half spectra, phase of the x grid, store
  for (int t = threadIdx.x; t < H * NL; t += NT) {
    const int l = t / H, k = t - l * H;
    if (l0 + l >= nlines) continue;
    const C zk = buf[k * PT + l];
    const C zc = cconj(buf[((L - k) % L) * PT + l]);
    C A = cscale(cadd(zk, zc), 0.5f);
    C B = cscale(cmul_mi(csub(zk, zc)), 0.5f);
    if (grid == 0) {
      const C ph = phs[k];
      A = cmul(A, ph);
      B = cmul(B, ph);
    }
    const int y0 = 2 * (l0 + l);
    C* o = out + (((int64_t)b * 3 + grid) * g.Lz + z) * ((int64_t)g.Ly * H);
    o[(int64_t)y0 * H + k] = A;
    if (y0 + 1 < g.Ly) o[(int64_t)(y0 + 1) * H + k] = B;
  }
}

template <int R1, int R2, int R3, int NL, int NT>
__global__ void __launch_bounds__(NT) k_xinv_fast(XArgs a, const C* __restrict__ in, const float* __restrict__ x,
                                                  float* __restrict__ y, const C* __restrict__ stw, int twn,
                                                  int off2, int off3, const C* __restrict__ phx) {
  using P = fast::Plan<R1, R2, R3>;
  constexpr int L = P::L, H = L / 2 + 1, PT = NL + 1;
  constexpr int BUFN = L * PT > 2 * NL * H ? L * PT : 2 * NL * H;   // the transform, or the raw rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tws = buf + BUFN;
  C* phs = tws + twn;                 // half-voxel phases of the x grid
  fast::load_table<NT>(tws, stw, twn);
  fast::load_table<NT>(phs, phx, H);
  const Geom& g = a.g;
  const int z = blockIdx.y;
  const int bo = blockIdx.z;                 // b * 3 + orientation
  const int al = bo % 3, b = bo / 3;
  const int s = b / a.nrhs, r = b % a.nrhs;
  const int l0 = blockIdx.x * NL;
  const int64_t plane = (int64_t)g.Ly * H;
  const C* srcA = in + (((int64_t)b * 6 + al) * g.Lz + z) * plane;        // potential
  const C* srcB = in + (((int64_t)b * 6 + 3 + al) * g.Lz + z) * plane;    // field
  // the potential and field half spectra of the tile's rows (each a
  // contiguous run of nl H values) into the buffer by cp.async, every copy in
  // flight at once: potential at buf[l H + k], field at buf[(NL + l) H + k]
  const int nl = min(NL, g.Ly - l0);
  // row starts of the tile's rows, for the gather
  __shared__ int rs[2][NL + 1];
  const int64_t row0 = ((int64_t)al * g.Lz + z) * g.Ly + l0;
  for (int i = threadIdx.x; i < 2 * (nl + 1); i += NT) {
    const int kind = i / (nl + 1), k = i - kind * (nl + 1);
    rs[kind][k] = a.rstart[(2 * (int64_t)s + kind) * a.R + row0 + k];
  }
  for (int e = threadIdx.x; e < nl * H; e += NT) {
    fast::cp_async8(&buf[e], srcA + (int64_t)l0 * H + e);
    fast::cp_async8(&buf[NL * H + e], srcB + (int64_t)l0 * H + e);
  }
  fast::cp_async_commit();
  fast::cp_async_wait_all();
  __syncthreads();                                                        // tables and rows loaded
  // Hermitian extension of potential + i field, built by the first stage as
  // it reads (value k gives line entries k and L - k)
  fast::transform_inplace_ld<P, NL, NT, true, PT, false, true>(buf, tws, off2, off3, [&](int l, int pos) -> C {
    if (l >= nl) return mk<C>(0.f, 0.f);
    const int k = pos <= L / 2 ? pos : L - pos;
    C A = buf[l * H + k], B = buf[(NL + l) * H + k];
    if (al == 0) {
      const C ph = cconj(phs[k]);
      A = cmul(A, ph);
      B = cmul(B, ph);
    }
    if (pos > L / 2) {
      A = cconj(A);
      B = cconj(B);
    }
    return cadd(A, cmul_pi(B));
  });
  // gather at the panels of the tile's rows (consecutive in the canonical
  // order: one contiguous range per kind), threads over the panels, a
  // panel's row by bisection of the row starts
  const float* xr = x + (int64_t)r * a.N;
  float* yr = y + (int64_t)r * a.N;
#pragma unroll
  for (int kind = 0; kind < 2; ++kind) {
    const int* rk = rs[kind];
    for (int p = rk[0] + threadIdx.x; p < rk[nl]; p += NT) {
      int lo = 0, hi = nl;                      // rk[lo] <= p < rk[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rk[mid] <= p) lo = mid;
        else hi = mid;
      }
      const C v = buf[a.px[p] * PT + lo];
      yr[p] = kind == 0 ? v.x : a.idiag[p] * xr[p] + v.y;   // conductor: potential; dielectric: Eq. 4
    }
  }
}

XArgs xargs(const Handle& h, int nrhs) {
  XArgs a;
  a.g = h.g;
  a.nrhs = nrhs;
  a.N = h.pan.N;
  a.rstart = h.pan.rstart.p;
  a.px = h.pan.px.p;
  a.idiag = h.pan.idiag_f.p;
  a.R = 3 * (int64_t)h.g.Lz * h.g.Ly;
  return a;
}

template <int R1, int R2, int R3, int NL, int NT>
int launch_xfwd(const Handle& h, const float* x, C* out, int nrhs, cudaStream_t st) {
  const Geom& g = h.g;
  const Plan1D<float2>& p = h.pf[0];
  constexpr int L = R1 * R2 * R3;
  const size_t sm = ((size_t)L * (NL + 1) + p.twn + L / 2 + 1) * sizeof(C);
  VC_CHECK(2 * g.Lx <= L, VOXCAP_ERR_UNSUPPORTED, "x padding shorter than twice the grid");
  auto kern = k_xfwd_fast<R1, R2, R3, NL, NT>;
  VC_TRY(set_smem(kern, sm));
  const int nlines = (g.Ly + 1) / 2;
  const int B = h.pan.S * nrhs;
  dim3 grid((nlines + NL - 1) / NL, g.Lz, B * 3);
  kern<<<grid, NT, sm, st>>>(xargs(h, nrhs), x, out, p.stw, p.twn, p.twoff[1], p.nst >= 3 ? p.twoff[2] : 0,
                             h.phf[0]);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

template <int R1, int R2, int R3, int NL, int NT>
int launch_xinv(const Handle& h, const C* in, const float* x, float* y, int nrhs, cudaStream_t st) {
  const Geom& g = h.g;
  const Plan1D<float2>& p = h.pf[0];
  constexpr int L = R1 * R2 * R3, H = L / 2 + 1;
  constexpr int BUFN = L * (NL + 1) > 2 * NL * H ? L * (NL + 1) : 2 * NL * H;
  const size_t sm = ((size_t)BUFN + p.twn + H) * sizeof(C);
  VC_CHECK(2 * g.Lx <= L, VOXCAP_ERR_UNSUPPORTED, "x padding shorter than twice the grid");
  auto kern = k_xinv_fast<R1, R2, R3, NL, NT>;
  VC_TRY(set_smem(kern, sm));
  const int B = h.pan.S * nrhs;
  dim3 grid((g.Ly + NL - 1) / NL, g.Lz, B * 3);
  kern<<<grid, NT, sm, st>>>(xargs(h, nrhs), in, x, y, p.stw, p.twn, p.twoff[1], p.nst >= 3 ? p.twoff[2] : 0,
                             h.phf[0]);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

// plan -> instantiation; fwd selects xfwd or xinv
template <bool FWD>
int dispatch_x(const Handle& h, const float* x, const C* in, C* out, float* y, int nrhs, cudaStream_t st) {
  const Plan1D<float2>& p = h.pf[0];
  const int* r = p.radix;
#define VC_X(A, B_, C_, NL, NT)                                                                  \
  return FWD ? launch_xfwd<A, B_, C_, NL, NT>(h, x, out, nrhs, st)                               \
             : launch_xinv<A, B_, C_, NL, NT>(h, in, x, y, nrhs, st)
  if (p.nst == 2) {
    if (r[0] == 4 && r[1] == 9) VC_X(4, 9, 1, 16, 128);
    if (r[0] == 8 && r[1] == 9) VC_X(8, 9, 1, 16, 128);
    if (r[0] == 16 && r[1] == 9) VC_X(16, 9, 1, 16, 256);
  } else if (p.nst == 3 && r[2] == 9) {
    if (r[0] == 8 && r[1] == 4) VC_X(8, 4, 9, 16, 256);
    if (r[0] == 16 && r[1] == 4) VC_X(16, 4, 9, 16, 256);
    if (r[0] == 16 && r[1] == 8) VC_X(16, 8, 9, 16, 576);
  }
#undef VC_X
  set_error("no compiled x-pass plan for this length");
  return VOXCAP_ERR_UNSUPPORTED;
}

}  // namespace

bool fast_x_ok(const Handle& h) { return fast_plan_ok(h.pf[0]); }

int fast_xfwd(const Handle& h, const float* x, float2* out, int nrhs, cudaStream_t st) {
  return dispatch_x<true>(h, x, nullptr, out, nullptr, nrhs, st);
}

int fast_xinv(const Handle& h, const float2* in, const float* x, float* y, int nrhs, cudaStream_t st) {
  return dispatch_x<false>(h, x, in, nullptr, y, nrhs, st);
}

}  // namespace vc
