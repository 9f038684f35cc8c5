// Block-circulant embedding of the Toeplitz tensors and their FFT
// (Eqs. 11-12, Appendix B), plus the FFT plans shared with the products.
//
// Frame.  Shifting every face grid by half a voxel along its own normal puts
// all panel centres on the voxel-centre lattice.  In that frame each kernel
// is even or odd about 0 along every axis, so its spectrum is real (P) or
// imaginary (E):
//     K^{ab}(k) = exp(-i pi k_a/M_a) * S^{ab}(k) * exp(+i pi k_b/M_b),
//     S = R (potential blocks)  or  S = -i R (normal-field blocks),
// with R real and R(M-k) = +-R(k) along each axis.  Only R on the octant
// [0,M_x/2] x [0,M_y/2] x [0,M_z/2] is stored, FP64 and FP32, scaled by
// 1/(M_x M_y M_z).  The products apply the half-voxel phases to the charge
// spectra (exp(+i pi k_b/M_b) on grid b) and to the results
// (exp(-i pi k_a/M_a) on grid a).  P^{yx}, P^{zx}, P^{zy} are the same real R
// as P^{xy}, P^{xz}, P^{yz}: this is Eq. 12 in the shifted frame.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fast.cuh"
#include "internal.h"

namespace vc {

// ------------------------------------------------------------ padding / plans
static bool smooth7(int n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Padded length along an axis: the paper's 2(N+1) (mode 1), or the cheapest
// even 2/3/5/7-smooth length >= 2N+1 within 25% of it by the FFT cost model.
static int pick_length(int N, int mode) {
  if (mode == 1) return 2 * (N + 1);
  int lo = 2 * N + 1;
  if (lo & 1) ++lo;
  if (mode == 2) {                       // smallest even smooth length
    while (!smooth7(lo)) lo += 2;
    return lo;
  }
  int best = -1;
  double bc = 1e300;
  for (int m = lo; m <= lo + lo / 4 + 2; m += 2) {
    if (!smooth7(m)) continue;
    const double c = fft_cost(m);
    if (c < bc) { bc = c; best = m; }
  }
  if (best < 0) {
    best = lo;
    while (!smooth7(best)) best += 2;
  }
  return best;
}

// cos and sin of 2 pi m / n in double, the angle reduced exactly in integers
// to at most pi/4 before the library call (about one ulp at any m, n).
static void unit_root(int64_t m, int64_t n, double* c, double* s) {
  const double half_pi = 1.57079632679489661923132169163975144;
  int64_t a = (4 * m) % (4 * n);                    // angle = (pi/2) a / n
  if (a < 0) a += 4 * n;
  const int q = (int)(a / n);                       // quadrant
  const int64_t r = a - (int64_t)q * n;             // within-quadrant angle (pi/2) r / n
  double sp, cp;                                    // sin, cos of the within-quadrant angle
  if (2 * r <= n) {
    const double t = half_pi * (double)r / (double)n;
    sp = std::sin(t);
    cp = std::cos(t);
  } else {
    const double t = half_pi * (double)(n - r) / (double)n;
    sp = std::cos(t);
    cp = std::sin(t);
  }
  switch (q) {
    case 0: *c = cp; *s = sp; break;
    case 1: *c = -sp; *s = cp; break;
    case 2: *c = -cp; *s = -sp; break;
    default: *c = sp; *s = -cp; break;
  }
}

// Stage twiddles of a radix plan (see Plan1D) and the half-voxel phases
// exp(+i pi m / L).
template <typename C>
static void fill_tables(std::vector<C>& stw, std::vector<C>& ph, int L, const int* radix, int nst,
                        int* Ns, int* twoff) {
  stw.clear();
  int ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = radix[s];
    Ns[s] = ns;
    twoff[s] = (int)stw.size();
    for (int k = 0; k < ns; ++k)
      for (int r = 1; r < R; ++r) {
        double cr, si;
        unit_root(-(int64_t)r * k, (int64_t)ns * R, &cr, &si);     // exp(-2 pi i r k / (ns R))
        C c;
        c.x = (decltype(C::x))cr;
        c.y = (decltype(C::x))si;
        stw.push_back(c);
      }
    ns *= R;
  }
  ph.resize(L);
  for (int m = 0; m < L; ++m) {
    double cr, si;
    unit_root(m, 2 * (int64_t)L, &cr, &si);                      // exp(+i pi m / L)
    ph[m].x = (decltype(C::x))cr;
    ph[m].y = (decltype(C::x))si;
  }
}

// Host staging of the plan tables: each table starts on a 16-byte boundary.
struct TableStage {
  std::vector<char> bytes;
  template <typename C> size_t put(const std::vector<C>& v) {
    const size_t off = (bytes.size() + 15) / 16 * 16;
    bytes.resize(off + std::max<size_t>(v.size(), 1) * sizeof(C));
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(C));
    return off;
  }
};

// Fill the FP64/FP32 plans of one radix order and stage their twiddles (and
// the phases, when asked); the offsets into the staged table come back.
static void make_plan(int L, const int* rad, int nst, TableStage& ts, Plan1D<double2>& pd,
                      Plan1D<float2>& pf, size_t* off_d, size_t* off_f, size_t* ph_d, size_t* ph_f) {
  int Ns[kMaxStages], twoff[kMaxStages];
  std::vector<double2> twd, phd;
  std::vector<float2> twf, phf;
  fill_tables(twd, phd, L, rad, nst, Ns, twoff);
  fill_tables(twf, phf, L, rad, nst, Ns, twoff);
  *off_d = ts.put(twd);
  *off_f = ts.put(twf);
  if (ph_d) {
    *ph_d = ts.put(phd);
    *ph_f = ts.put(phf);
  }
  pd.L = pf.L = L;
  pd.nst = pf.nst = nst;
  pd.twn = pf.twn = (int)twd.size();
  for (int s = 0; s < nst; ++s) {
    pd.radix[s] = pf.radix[s] = rad[s];
    pd.Ns[s] = pf.Ns[s] = Ns[s];
    pd.fNs[s] = pf.fNs[s] = make_fastdiv((uint32_t)Ns[s]);
    pd.twoff[s] = pf.twoff[s] = twoff[s];
  }
}

int build_fft_plans(Handle& h) {
  Geom& g = h.g;
  int n[3] = {g.nx, g.ny, g.nz};
  int M[3];
  TableStage ts;
  size_t off[3][6], zoff[2][4];
  for (int a = 0; a < 3; ++a) {
    M[a] = pick_length(n[a], h.opts.pad_mode);
    int rad[kMaxStages], nst = 0;
    VC_CHECK(factor_length(M[a], rad, &nst), VOXCAP_ERR_UNSUPPORTED,
             "FFT length " + std::to_string(M[a]) + " is not 2/3/5/7-smooth (use pad_mode 0)");
    int zord[2][kMaxStages], zn[2] = {nst, nst};
    if (a == 2) {
      // the z pass keeps its last forward radix in registers: order 0 puts the
      // largest radix <= 9 last, order 1 the smallest (more threads per tile);
      // a last 16 (too many registers per line and grid) is split into 4 x 4
      for (int v = 0; v < 2; ++v) {
        for (int s = 0; s < nst; ++s) zord[v][s] = rad[s];
        int best = -1;
        for (int s = 0; s < nst; ++s) {
          const int R = zord[v][s];
          if (v == 0 ? (R <= 9 && (best < 0 || R > zord[v][best])) : (best < 0 || R < zord[v][best])) best = s;
        }
        if (best < 0) best = 0;
        std::swap(zord[v][best], zord[v][nst - 1]);
        if (zord[v][nst - 1] == 16) {
          zord[v][nst - 1] = 4;
          zord[v][zn[v]++] = 4;
        }
      }
      for (int s = 0; s < zn[0]; ++s) rad[s] = zord[0][s];
      nst = zn[0];
    }
    make_plan(M[a], rad, nst, ts, h.pd[a], h.pf[a], &off[a][0], &off[a][1], &off[a][2], &off[a][3]);
    int rev[kMaxStages];
    for (int s = 0; s < nst; ++s) rev[s] = rad[nst - 1 - s];
    make_plan(M[a], rev, nst, ts, h.pdr[a], h.pfr[a], &off[a][4], &off[a][5], nullptr, nullptr);
    if (a == 2) {
      h.nzvar = 1;
      bool same = zn[1] == zn[0];
      for (int s = 0; same && s < zn[0]; ++s) same = zord[1][s] == zord[0][s];
      if (!same) h.nzvar = 2;
      for (int v = 0; v < h.nzvar; ++v) {
        int r2[kMaxStages];
        for (int s = 0; s < zn[v]; ++s) r2[s] = zord[v][zn[v] - 1 - s];
        make_plan(M[a], zord[v], zn[v], ts, h.pzd[v], h.pzf[v], &zoff[v][0], &zoff[v][1], nullptr, nullptr);
        make_plan(M[a], r2, zn[v], ts, h.pzdr[v], h.pzfr[v], &zoff[v][2], &zoff[v][3], nullptr, nullptr);
      }
    }
  }
  VC_TRY(h.plan_tab.alloc(ts.bytes.size()));
  // from pageable memory: returns once the bytes are staged, so `ts` may go
  VC_CUDA(cudaMemcpyAsync(h.plan_tab.p, ts.bytes.data(), ts.bytes.size(), cudaMemcpyHostToDevice, h.stream));
  char* base = h.plan_tab.p;
  for (int a = 0; a < 3; ++a) {
    h.pd[a].stw = reinterpret_cast<const double2*>(base + off[a][0]);
    h.pf[a].stw = reinterpret_cast<const float2*>(base + off[a][1]);
    h.phd[a] = reinterpret_cast<const double2*>(base + off[a][2]);
    h.phf[a] = reinterpret_cast<const float2*>(base + off[a][3]);
    h.pdr[a].stw = reinterpret_cast<const double2*>(base + off[a][4]);
    h.pfr[a].stw = reinterpret_cast<const float2*>(base + off[a][5]);
  }
  for (int v = 0; v < h.nzvar; ++v) {
    h.pzd[v].stw = reinterpret_cast<const double2*>(base + zoff[v][0]);
    h.pzf[v].stw = reinterpret_cast<const float2*>(base + zoff[v][1]);
    h.pzdr[v].stw = reinterpret_cast<const double2*>(base + zoff[v][2]);
    h.pzfr[v].stw = reinterpret_cast<const float2*>(base + zoff[v][3]);
  }
  h.zvar = 0;
  h.ztx = -1;
  g.Mx = M[0]; g.My = M[1]; g.Mz = M[2];
  g.Hx = g.Mx / 2 + 1;
  g.Oy = g.My / 2 + 1;
  g.Oz = g.Mz / 2 + 1;
  return VOXCAP_OK;
}

// ------------------------------------------------------------ embedding
// Per-axis mapping of a circulant index to the Toeplitz index and sign.
struct AxisMap {
  int type;   // 0 even@0, 1 odd@0, 2 even@+1/2, 3 odd@+1/2, 4 even@-1/2
  int dmin, dmax, M;
};

__device__ __forceinline__ bool axis_lookup(const AxisMap& am, int i, int* e, double* sg) {
  int d;
  if (i <= am.dmax) d = i;
  else if (i >= am.M + am.dmin) d = i - am.M;
  else return false;
  switch (am.type) {
    case 0: *e = d < 0 ? -d : d; break;
    case 1: *e = d < 0 ? -d : d; if (d < 0) *sg = -*sg; break;
    case 2: *e = d >= 1 ? d - 1 : -d; break;
    case 3: *e = d >= 1 ? d - 1 : -d; if (d < 1) *sg = -*sg; break;
    default: *e = d >= 0 ? d : -d - 1; break;
  }
  return true;
}

// tables and index maps of the 15 kernels
struct EmbedSet {
  const double* T[kNumKernels];
  int tx[kNumKernels], ty[kNumKernels];
  AxisMap ax[kNumKernels], ay[kNumKernels], az[kNumKernels];
};

// circ[b] = circulant embedding of kernel k0 + b (b = blockIdx.y)
template <typename T>
__global__ void k_embed(EmbedSet es, int k0, int64_t Mtot, T* __restrict__ circ) {
  const int b = blockIdx.y, kk = k0 + b;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Mtot) return;
  const AxisMap& ax = es.ax[kk];
  const AxisMap& ay = es.ay[kk];
  const AxisMap& az = es.az[kk];
  const int i = (int)(t % ax.M), j = (int)((t / ax.M) % ay.M), k = (int)(t / ((int64_t)ax.M * ay.M));
  int ex, ey, ez;
  double sg = 1.0;
  double v = 0.0;
  if (axis_lookup(ax, i, &ex, &sg) && axis_lookup(ay, j, &ey, &sg) && axis_lookup(az, k, &ez, &sg))
    v = sg * es.T[kk][(int64_t)ex + (int64_t)es.tx[kk] * (ey + (int64_t)es.ty[kk] * ez)];
  circ[(int64_t)b * Mtot + t] = (T)v;
}

static AxisMap axis_map(int kk, int a, int N, int M) {
  const int te = ker_test(kk), so = ker_src(kk);
  const bool E = kk >= 6;
  AxisMap am;
  am.M = M;
  if (te == so) {
    if (a == te) { am.type = E ? 1 : 0; am.dmin = -N; am.dmax = N; }
    else { am.type = 0; am.dmin = -(N - 1); am.dmax = N - 1; }
  } else if (a == te) {
    am.type = E ? 3 : 2; am.dmin = -(N - 1); am.dmax = N;
  } else if (a == so) {
    am.type = 4; am.dmin = -N; am.dmax = N - 1;
  } else {
    am.type = 0; am.dmin = -(N - 1); am.dmax = N - 1;
  }
  return am;
}

// ------------------------------------------------------------ generic FFT passes
// Real rows of length M (x) -> half spectra (Hx), two rows per complex line.
template <typename T, int NL>
__global__ void k_rows_r2c(const T* __restrict__ in, int64_t nrows, int M, int H,
                           C_t<T>* __restrict__ out, Plan1D<C_t<T>> plan) {
  using C = C_t<T>;
  extern __shared__ unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* scr = buf + (size_t)M * NL;
  C* stw = scr + (size_t)M * NL;
  load_twiddles(stw, plan);
  const int64_t row0 = (int64_t)blockIdx.x * NL * 2;
  for (int t = threadIdx.x; t < M * NL; t += blockDim.x) {
    int l = t % NL, x = t / NL;
    int64_t ra = row0 + 2 * l, rb = ra + 1;
    T a = ra < nrows ? in[ra * M + x] : (T)0;
    T b = rb < nrows ? in[rb * M + x] : (T)0;
    buf[x * NL + l] = mk<C>(a, b);
  }
  __syncthreads();
  C* res = fft_lines<NL>(buf, scr, NL, plan, stw, false);
  for (int t = threadIdx.x; t < H * NL; t += blockDim.x) {
    int l = t % NL, k = t / NL;
    int64_t ra = row0 + 2 * l, rb = ra + 1;
    C z = res[k * NL + l];
    C zc = cconj(res[((M - k) % M) * NL + l]);
    C A = cscale(cadd(z, zc), (T)0.5);
    C B = cscale(cmul_mi(csub(z, zc)), (T)0.5);
    if (ra < nrows) out[ra * H + k] = A;
    if (rb < nrows) out[rb * H + k] = B;
  }
}

// In-place complex FFT along a strided axis of a [outer][L][inner] array;
// each block handles TX consecutive inner positions of one outer index.
template <typename T, int TX>
__global__ void k_strided_c2c(C_t<T>* __restrict__ data, int64_t outer, int L, int64_t inner,
                              Plan1D<C_t<T>> plan, bool inv) {
  using C = C_t<T>;
  extern __shared__ unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* scr = buf + (size_t)L * TX;
  C* stw = scr + (size_t)L * TX;
  load_twiddles(stw, plan);
  const int64_t tiles = (inner + TX - 1) / TX;
  const int64_t o = blockIdx.x / tiles;
  const int64_t i0 = (blockIdx.x % tiles) * TX;
  C* base = data + o * L * inner;
  for (int t = threadIdx.x; t < L * TX; t += blockDim.x) {
    int c = t % TX, p = t / TX;
    int64_t ii = i0 + c;
    buf[p * TX + c] = ii < inner ? base[(int64_t)p * inner + ii] : mk<C>((T)0, (T)0);
  }
  __syncthreads();
  C* res = fft_lines<TX>(buf, scr, TX, plan, stw, inv);
  for (int t = threadIdx.x; t < L * TX; t += blockDim.x) {
    int c = t % TX, p = t / TX;
    int64_t ii = i0 + c;
    if (ii < inner) base[(int64_t)p * inner + ii] = res[p * TX + c];
  }
}

// Extract the real octant R of kernel k0 + b (b = blockIdx.y) from its
// half spectrum (see file comment); phases and scaling in FP64.
template <typename T>
__global__ void k_extract(const C_t<T>* __restrict__ spec, int64_t Htot, Geom g, int k0,
                          const double2* __restrict__ phx, const double2* __restrict__ phy,
                          const double2* __restrict__ phz, double scale,
                          double* __restrict__ Rd, float* __restrict__ Rf, float* __restrict__ Rb) {
  const int b = blockIdx.y, kk = k0 + b;
  const int te = ker_test(kk), so = ker_src(kk);
  const bool E = kk >= 6;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)g.Hx * g.Oy * g.Oz;
  if (t >= n) return;
  const int kx = (int)(t % g.Hx), ky = (int)((t / g.Hx) % g.Oy), kz = (int)(t / ((int64_t)g.Hx * g.Oy));
  const C_t<T> w = spec[(int64_t)b * Htot + ((int64_t)kz * g.My + ky) * g.Hx + kx];
  double2 v = make_double2((double)w.x, (double)w.y);
  // undo exp(-i pi k_te/M) S exp(+i pi k_so/M):  multiply by exp(+i pi k_te/M) exp(-i pi k_so/M)
  if (te != so) {
    const double2* pt = te == 0 ? phx : (te == 1 ? phy : phz);
    const double2* ps = so == 0 ? phx : (so == 1 ? phy : phz);
    const int kt = te == 0 ? kx : (te == 1 ? ky : kz);
    const int ks = so == 0 ? kx : (so == 1 ? ky : kz);
    v = cmul(v, pt[kt]);
    v = cmul(v, cconj(ps[ks]));
  }
  double r = E ? -v.y : v.x;     // S = -i R  ->  R = i S;  Re(i S) = -Im(S)
  r *= scale;
  Rd[kk * n + t] = r;
  Rf[kk * n + t] = (float)r;
  if (Rb) {
    const int nm = (g.Hx + kSpecBlk - 1) / kSpecBlk, m = kx / kSpecBlk;
    Rb[((((int64_t)ky * nm + m) * g.Oz + kz) * kNumKernels + kk) * kSpecBlk + kx % kSpecBlk] = (float)r;
  }
}

// largest power-of-two line count (<= maxlines) whose two buffers fit in 96 KB
template <typename T> static int smem_limit_lines(int L, int maxlines) {
  const size_t budget = 96 * 1024;
  int nl = (int)(budget / (2 * (size_t)L * sizeof(C_t<T>)));
  int p = 1;
  while (p * 2 <= nl && p * 2 <= maxlines) p *= 2;
  return p;
}

// The spectra of kernels in batches that fit a 512 MB scratch budget, with
// transforms in T (FP64, or FP32 when the entries themselves are only
// FP32-accurate: the FP64 copy is then the FP32 spectrum widened).
template <typename T>
static int spectra_impl(Handle& h) {
  using C = C_t<T>;
  const Geom& g = h.g;
  const int n[3] = {g.nx, g.ny, g.nz};
  const int64_t Mtot = (int64_t)g.Mx * g.My * g.Mz;
  const int64_t Htot = (int64_t)g.Hx * g.My * g.Mz;
  const int64_t Otot = (int64_t)g.Hx * g.Oy * g.Oz;
  const size_t per_kernel = (size_t)Mtot * sizeof(T) + (size_t)Htot * sizeof(C);
  const int nb = (int)std::max<size_t>(1, std::min<size_t>(kNumKernels, ((size_t)512 << 20) / per_kernel));
  DBuf<T> circ;
  DBuf<C> spec;
  VC_TRY(circ.alloc((size_t)Mtot * nb));
  VC_TRY(spec.alloc((size_t)Htot * nb));
  VC_TRY(h.spec_d.alloc((size_t)Otot * kNumKernels));
  VC_TRY(h.spec_f.alloc((size_t)Otot * kNumKernels));
  float* blocked = nullptr;
  if (fast_z_ok(h)) {
    const size_t nblk = (size_t)g.Oy * ((g.Hx + kSpecBlk - 1) / kSpecBlk) * g.Oz * kNumKernels * kSpecBlk;
    VC_TRY(h.spec_fb.alloc(nblk));
    VC_CUDA(cudaMemsetAsync(h.spec_fb.p, 0, nblk * sizeof(float), h.stream));
    blocked = h.spec_fb.p;
  }
  EmbedSet es;
  for (int kk = 0; kk < kNumKernels; ++kk) {
    es.T[kk] = h.toep[kk].p;
    es.tx[kk] = h.tdims[kk][0];
    es.ty[kk] = h.tdims[kk][1];
    es.ax[kk] = axis_map(kk, 0, n[0], g.Mx);
    es.ay[kk] = axis_map(kk, 1, n[1], g.My);
    es.az[kk] = axis_map(kk, 2, n[2], g.Mz);
  }
  const double scale = 1.0 / (double)Mtot;
  const int TB = 256;
  const Plan1D<C>& px = plan_of<T>(h, 0);
  const Plan1D<C>& py = plan_of<T>(h, 1);
  const Plan1D<C>& pz = plan_of<T>(h, 2);
  for (int k0 = 0; k0 < kNumKernels; k0 += nb) {
    const int nk = std::min(nb, kNumKernels - k0);
    k_embed<T><<<dim3((unsigned)((Mtot + TB - 1) / TB), nk), TB, 0, h.stream>>>(es, k0, Mtot, circ.p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
    // x: real rows -> half spectra
    {
      const int NL = smem_limit_lines<T>(g.Mx, 16);
      const int64_t nrows = (int64_t)nk * g.My * g.Mz;
      const unsigned nblk = (unsigned)((nrows + 2 * NL - 1) / (2 * NL));
      const size_t sm = (2 * (size_t)g.Mx * NL + px.twn) * sizeof(C);
#define VC_R2C(W)                                                                                  \
  VC_TRY(set_smem(k_rows_r2c<T, W>, sm));                                                          \
  k_rows_r2c<T, W><<<nblk, 256, sm, h.stream>>>(circ.p, nrows, g.Mx, g.Hx, spec.p, px);
      VC_TILE_DISPATCH(NL, VC_R2C)
#undef VC_R2C
      ::vc::note_launch();
      VC_CUDA(cudaGetLastError());
    }
    // y: [nk Mz][My][Hx] along My
    {
      const int TX = smem_limit_lines<T>(g.My, 16);
      const int64_t tiles = (g.Hx + TX - 1) / TX;
      const size_t sm = (2 * (size_t)g.My * TX + py.twn) * sizeof(C);
#define VC_C2CY(W)                                                                                  \
  VC_TRY(set_smem(k_strided_c2c<T, W>, sm));                                                        \
  k_strided_c2c<T, W><<<(unsigned)((int64_t)nk * g.Mz * tiles), 256, sm, h.stream>>>(spec.p, (int64_t)nk * g.Mz, \
                                                                                    g.My, g.Hx, py, false);
      VC_TILE_DISPATCH(TX, VC_C2CY)
#undef VC_C2CY
      ::vc::note_launch();
      VC_CUDA(cudaGetLastError());
    }
    // z: [nk][Mz][My*Hx] along Mz
    {
      const int TX = smem_limit_lines<T>(g.Mz, 16);
      const int64_t inner = (int64_t)g.My * g.Hx;
      const int64_t tiles = (inner + TX - 1) / TX;
      const size_t sm = (2 * (size_t)g.Mz * TX + pz.twn) * sizeof(C);
#define VC_C2CZ(W)                                                                                  \
  VC_TRY(set_smem(k_strided_c2c<T, W>, sm));                                                        \
  k_strided_c2c<T, W><<<(unsigned)(nk * tiles), 256, sm, h.stream>>>(spec.p, nk, g.Mz, inner, pz, false);
      VC_TILE_DISPATCH(TX, VC_C2CZ)
#undef VC_C2CZ
      ::vc::note_launch();
      VC_CUDA(cudaGetLastError());
    }
    k_extract<T><<<dim3((unsigned)((Otot + TB - 1) / TB), nk), TB, 0, h.stream>>>(
        spec.p, Htot, g, k0, h.phd[0], h.phd[1], h.phd[2], scale, h.spec_d.p, h.spec_f.p, blocked);
    ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  return VOXCAP_OK;
}

int build_spectra(Handle& h) { return h.far32 ? spectra_impl<float>(h) : spectra_impl<double>(h); }

}  // namespace vc
