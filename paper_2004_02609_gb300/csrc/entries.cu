// Block-Toeplitz tensors of Eqs. 5-6 (Appendix A-B), evaluated in FP64.
//
// Every one of the 15 tensors is one of four functions of the centre
// difference of the two unit panels, up to an axis permutation:
//   Ppar(h,s,t), Epar = dPpar/dh   parallel panels, normal offset h, in-plane s,t
//   Port(a,b,c), Eort = dPort/da   orthogonal panels; a along the test normal,
//                                  b along the source normal, c along the shared axis
// (normalised units, 1/(4 pi) included).
//
// Near field (panels within one voxel of each other): exact corner sums of
// 4-D antiderivatives of 1/r (the second difference of the panel-overlap
// triangle along shared axes, first differences along the others).  The
// normal-derivative closed forms play the role of the paper's Eqs. 15-16.
// Far field: the same integrals reduced to 2-D (parallel) or 3-D (orthogonal)
// integrals with triangle weights, by tensor Gauss-Legendre quadrature whose
// order falls with the gap between the panels.
#include <cmath>
#include <vector>

#include "internal.h"

namespace vc {

constexpr int kMaxGL = 10;
__constant__ double c_glx[kMaxGL + 1][kMaxGL];
__constant__ double c_glw[kMaxGL + 1][kMaxGL];

// Gauss-Legendre nodes / weights on [-1,1] by Newton iteration on P_n.
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static int ensure_gl_tables() {
  int dev = 0;
  VC_CUDA(cudaGetDevice(&dev));
  static bool done[64] = {false};
  if (dev < 64 && done[dev]) return VOXCAP_OK;
  double hx[kMaxGL + 1][kMaxGL] = {};
  double hw[kMaxGL + 1][kMaxGL] = {};
  for (int n = 1; n <= kMaxGL; ++n) gauss_legendre(n, hx[n], hw[n]);
  VC_CUDA(cudaMemcpyToSymbol(c_glx, hx, sizeof(hx)));
  VC_CUDA(cudaMemcpyToSymbol(c_glw, hw, sizeof(hw)));
  if (dev < 64) done[dev] = true;
  return VOXCAP_OK;
}

constexpr double kInv4Pi = 0.079577471545947667884441881686257181017229822870228;
__constant__ double c_cw[3] = {1.0, -2.0, 1.0};   // second difference at -1, 0, +1

// ln(a + sqrt(a^2 + rest2)), accurate for a < 0
__device__ __forceinline__ double logplus(double a, double rest2) {
  double r = sqrt(a * a + rest2);
  return a >= 0.0 ? log(a + r) : log(rest2 / (r - a));
}

// d^2/du^2 d^2/dv^2 F = 1/sqrt(u^2+v^2+h^2)
__device__ double F_par(double u, double v, double h) {
  double u2 = u * u, v2 = v * v, h2 = h * h;
  double r = sqrt(u2 + v2 + h2);
  double t = -(u2 + v2 - 2.0 * h2) * r * (1.0 / 6.0);
  double c1 = 0.5 * (u2 - h2) * v;
  if (c1 != 0.0) t += c1 * logplus(v, u2 + h2);
  double c2 = 0.5 * (v2 - h2) * u;
  if (c2 != 0.0) t += c2 * logplus(u, v2 + h2);
  if (h != 0.0 && u * v != 0.0) t -= u * v * h * atan(u * v / (h * r));
  return t;
}

// d^2/du^2 d^2/dv^2 Fh = -h / r^3  (h != 0)
__device__ double Fh_par(double u, double v, double h) {
  double u2 = u * u, v2 = v * v, h2 = h * h;
  double r = sqrt(u2 + v2 + h2);
  double t = h * r;
  if (v != 0.0) t -= h * v * logplus(v, u2 + h2);
  if (u != 0.0) t -= h * u * logplus(u, v2 + h2);
  if (u * v != 0.0) t -= u * v * atan(u * v / (h * r));
  return t;
}

// d/dp d/dq d^2/dw^2 H = 1/sqrt(p^2+q^2+w^2)
__device__ double H_ort(double p, double q, double w) {
  double p2 = p * p, q2 = q * q, w2 = w * w;
  double r = sqrt(p2 + q2 + w2);
  double t = -p * q * r * (1.0 / 3.0);
  if (p * q * w != 0.0) t += p * q * w * logplus(w, p2 + q2);
  double c = q * (0.5 * w2 - q2 * (1.0 / 6.0));
  if (c != 0.0) t += c * logplus(p, q2 + w2);
  c = p * (0.5 * w2 - p2 * (1.0 / 6.0));
  if (c != 0.0) t += c * logplus(q, p2 + w2);
  if (w != 0.0) {
    if (q != 0.0) t -= 0.5 * w * q2 * atan(p * w / (q * r));
    if (p != 0.0) t -= 0.5 * w * p2 * atan(q * w / (p * r));
    if (p * q != 0.0) t -= w2 * w * (1.0 / 6.0) * atan(p * q / (w * r));
  }
  return t;
}

// d/dq d^2/dw^2 Hp = 1/r; equals dH/dp up to terms the corner sum cancels
__device__ double Hp_ort(double p, double q, double w) {
  double p2 = p * p, q2 = q * q, w2 = w * w;
  double r = sqrt(p2 + q2 + w2);
  double t = -0.5 * q * r;
  if (w * q != 0.0) t += w * q * logplus(w, p2 + q2);
  double c = 0.5 * (w2 - p2);
  if (c != 0.0) t += c * logplus(q, p2 + w2);
  if (w * p != 0.0) t -= w * p * atan(q * w / (p * r));
  return t;
}

// ---- near field: corner sums ----
__device__ double par_cf(bool E, double h, double s, double t) {
  if (E && h == 0.0) return 0.0;
  double acc = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double wgt = c_cw[i] * c_cw[j];
      double u = s + (i - 1), v = t + (j - 1);
      acc += wgt * (E ? Fh_par(u, v, h) : F_par(u, v, h));
    }
  return acc * kInv4Pi;
}

__device__ double ort_cf(bool E, double a, double b, double c) {
  double acc = 0.0;
  for (int s1 = -1; s1 <= 1; s1 += 2)
    for (int s2 = -1; s2 <= 1; s2 += 2)
      for (int j = 0; j < 3; ++j) {
        double wgt = (double)(s1 * s2) * c_cw[j];
        double p = a + 0.5 * s1, q = b + 0.5 * s2, w = c + (j - 1);
        acc += wgt * (E ? Hp_ort(p, q, w) : H_ort(p, q, w));
      }
  return acc * kInv4Pi;
}

// ---- far field: Gauss-Legendre on the triangle-weighted reduced integrals ----
__device__ int gl_order(double gap) {
  if (gap < 2.5) return 9;
  if (gap < 3.5) return 8;
  if (gap < 5.5) return 7;
  if (gap < 9.5) return 6;
  if (gap < 19.5) return 5;
  if (gap < 49.5) return 4;
  return 3;
}

// Ppar = (1/4pi) Int_{-1}^{1} Int_{-1}^{1} (1-|p|)(1-|q|) / sqrt((s+p)^2+(t+q)^2+h^2)
__device__ double par_gl(bool E, double h, double s, double t, int n) {
  double acc = 0.0;
  for (int sp = -1; sp <= 1; sp += 2)
    for (int i = 0; i < n; ++i) {
      double pp = 0.5 * (1.0 + c_glx[n][i]);
      double wp = 0.5 * c_glw[n][i] * (1.0 - pp);
      double X = s + sp * pp;
      double accq = 0.0;
      for (int sq = -1; sq <= 1; sq += 2)
        for (int j = 0; j < n; ++j) {
          double qq = 0.5 * (1.0 + c_glx[n][j]);
          double wq = 0.5 * c_glw[n][j] * (1.0 - qq);
          double Y = t + sq * qq;
          double r2 = X * X + Y * Y + h * h;
          double ir = rsqrt(r2);
          accq += wq * (E ? -h * ir * ir * ir : ir);
        }
      acc += wp * accq;
    }
  return acc * kInv4Pi;
}

// Port = (1/4pi) Int_{a-1/2}^{a+1/2} dp Int_{b-1/2}^{b+1/2} dq Int_{-1}^{1} (1-|w|) dw
//        / sqrt(p^2 + q^2 + (c+w)^2);  Eort = d/da of it.
__device__ double ort_gl(bool E, double a, double b, double c, int n) {
  double acc = 0.0;
  for (int j = 0; j < n; ++j) {
    double q = b + 0.5 * c_glx[n][j];
    double wq = 0.5 * c_glw[n][j];
    for (int sw = -1; sw <= 1; sw += 2)
      for (int k = 0; k < n; ++k) {
        double ww = 0.5 * (1.0 + c_glx[n][k]);
        double wgt = wq * 0.5 * c_glw[n][k] * (1.0 - ww);
        double Z = c + sw * ww;
        double base = q * q + Z * Z;
        if (E) {
          double p1 = a + 0.5, p0 = a - 0.5;
          double r1 = p1 * p1 + base, r0 = p0 * p0 + base;
          double i1 = rsqrt(r1), i0 = rsqrt(r0);
          acc += wgt * (i1 - i0);
        } else {
          double sp = 0.0;
          for (int i = 0; i < n; ++i) {
            double p = a + 0.5 * c_glx[n][i];
            double r2 = p * p + base;
            double ir = rsqrt(r2);
            sp += 0.5 * c_glw[n][i] * ir;
          }
          acc += wgt * sp;
        }
      }
  }
  return acc * kInv4Pi;
}

// canonical functions at non-negative arguments (a, b > 0 half-integers)
__device__ double ppar_e(bool E, double h, double s, double t) {
  double gap = fmax(h, fmax(s - 1.0, t - 1.0));
  if (gap <= 1.0) return par_cf(E, h, s, t);
  if (E && h == 0.0) return 0.0;
  return par_gl(E, h, s, t, gl_order(gap));
}

__device__ double port_e(bool E, double a, double b, double c) {
  double gap = fmax(a - 0.5, fmax(b - 0.5, c - 1.0));
  if (gap <= 1.0) return ort_cf(E, a, b, c);
  return ort_gl(E, a, b, c, gl_order(gap));
}

// Value of one kernel tensor at Toeplitz index e (see voxcap_toeplitz).
__device__ double toeplitz_value(int kk, int ex, int ey, int ez) {
  const bool E = kk >= 6;
  const int te = ker_test(kk), so = ker_src(kk);
  const int e[3] = {ex, ey, ez};
  if (te == so) {
    const int a1 = te == 0 ? 1 : 0, a2 = te == 2 ? 1 : 2;
    return ppar_e(E, (double)e[te], (double)e[a1], (double)e[a2]);
  }
  const int ga = 3 - te - so;
  return port_e(E, e[te] + 0.5, e[so] + 0.5, (double)e[ga]);
}

__global__ void k_toeplitz(int kk, int dx, int dy, int dz, double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)dx * dy * dz;
  if (t >= n) return;
  int ex = (int)(t % dx), ey = (int)((t / dx) % dy), ez = (int)(t / ((int64_t)dx * dy));
  out[t] = toeplitz_value(kk, ex, ey, ez);
}

void toeplitz_dims(const Geom& g, int kk, int* d) {
  const int te = ker_test(kk), so = ker_src(kk);
  const int n[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) d[a] = n[a];
  if (te == so) d[te] = n[te] + 1;
}

int build_toeplitz(Handle& h) {
  VC_TRY(ensure_gl_tables());
  for (int kk = 0; kk < kNumKernels; ++kk) {
    int* d = h.tdims[kk];
    toeplitz_dims(h.g, kk, d);
    int64_t n = (int64_t)d[0] * d[1] * d[2];
    VC_TRY(h.toep[kk].alloc((size_t)n));
    const int TB = 128;
    k_toeplitz<<<(unsigned)((n + TB - 1) / TB), TB, 0, h.stream>>>(kk, d[0], d[1], d[2],
                                                                     h.toep[kk].p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  return VOXCAP_OK;
}

// ---- arbitrary panel pairs ----
__global__ void k_entries(int n, const int32_t* __restrict__ kind, const int32_t* __restrict__ to,
                          const int32_t* __restrict__ so, const double* __restrict__ d,
                          double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool E = kind[i] != 0;
  const int te = to[i], sr = so[i];
  const double dd[3] = {d[3 * i], d[3 * i + 1], d[3 * i + 2]};
  double v;
  if (te == sr) {
    const int a1 = te == 0 ? 1 : 0, a2 = te == 2 ? 1 : 2;
    v = ppar_e(E, fabs(dd[te]), fabs(dd[a1]), fabs(dd[a2]));
    if (E && dd[te] < 0.0) v = -v;
  } else {
    const int ga = 3 - te - sr;
    v = port_e(E, fabs(dd[te]), fabs(dd[sr]), fabs(dd[ga]));
    if (E && dd[te] < 0.0) v = -v;
  }
  out[i] = v;
}

int entries_eval(int n, const int32_t* kind, const int32_t* to, const int32_t* so,
                 const double* d, double* out, cudaStream_t st) {
  VC_TRY(ensure_gl_tables());
  if (n <= 0) return VOXCAP_OK;
  const int TB = 128;
  k_entries<<<(n + TB - 1) / TB, TB, 0, st>>>(n, kind, to, so, d, out); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  VC_CUDA(cudaStreamSynchronize(st));
  return VOXCAP_OK;
}

}  // namespace vc
