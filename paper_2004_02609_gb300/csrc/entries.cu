// Block-Toeplitz tensors of Eqs. 5-6 (Appendix A-B): near field in FP64, far
// field in FP64 or, for the FP32-refinement set-up, with FP32 inner sums.
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
// FP32 forms for the far field: half-nodes x/2, half-weights w/2, the
// triangle-rule abscissae (1+x)/2 and weights (w/2)(1 - (1+x)/2)
__constant__ float c_fx[kMaxGL + 1][kMaxGL];
__constant__ float c_fw[kMaxGL + 1][kMaxGL];
__constant__ float c_fp[kMaxGL + 1][kMaxGL];
__constant__ float c_fq[kMaxGL + 1][kMaxGL];

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
  float fx[kMaxGL + 1][kMaxGL] = {}, fw[kMaxGL + 1][kMaxGL] = {};
  float fp[kMaxGL + 1][kMaxGL] = {}, fq[kMaxGL + 1][kMaxGL] = {};
  for (int n = 1; n <= kMaxGL; ++n)
    for (int i = 0; i < n; ++i) {
      const double pp = 0.5 * (1.0 + hx[n][i]);
      fx[n][i] = (float)(0.5 * hx[n][i]);
      fw[n][i] = (float)(0.5 * hw[n][i]);
      fp[n][i] = (float)pp;
      fq[n][i] = (float)(0.5 * hw[n][i] * (1.0 - pp));
    }
  VC_CUDA(cudaMemcpyToSymbol(c_fx, fx, sizeof(fx)));
  VC_CUDA(cudaMemcpyToSymbol(c_fw, fw, sizeof(fw)));
  VC_CUDA(cudaMemcpyToSymbol(c_fp, fp, sizeof(fp)));
  VC_CUDA(cudaMemcpyToSymbol(c_fq, fq, sizeof(fq)));
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
// Orders by the gap between the panels (in voxels), the smallest that keep
// the quadrature error below 2e-14 relative against the adaptive FP64
// integrals over sampled configurations at each gap.
__device__ int gl_order_par(double gap) {
  if (gap < 2.5) return 9;
  if (gap < 3.5) return 8;
  if (gap < 9.5) return 6;
  if (gap < 19.5) return 5;
  if (gap < 59.5) return 4;
  return 3;
}
__device__ int gl_order_ort(double gap) {
  if (gap < 3.5) return 7;
  if (gap < 5.5) return 6;
  if (gap < 19.5) return 5;
  if (gap < 49.5) return 4;
  return 3;
}

// ---- far field with FP32 sums ----
// The same rules with the inner sums in FP32 and the outer accumulation in
// FP64: entries to about 1e-7 relative, the accuracy of the FP32 products
// they feed.  Used when the set-up keeps FP64 for the near field only.
__device__ __forceinline__ float sqrt_approx(float x) { return x * rsqrtf(x); }

__device__ void par_pe_far32(double h, double s, double t, int n, double* P, double* E) {
  const float hf = (float)h, h2 = hf * hf;
  const float sf = (float)s, tf = (float)t;
  double ap = 0.0, ae = 0.0;
  for (int sp = -1; sp <= 1; sp += 2)
    for (int i = 0; i < n; ++i) {
      const float X = sf + (float)sp * c_fp[n][i];
      const float X2h = X * X + h2;
      float qp = 0.0f, qe = 0.0f;
      for (int sq = -1; sq <= 1; sq += 2)
        for (int j = 0; j < n; ++j) {
          const float Y = tf + (float)sq * c_fp[n][j];
          const float ir = rsqrtf(X2h + Y * Y);
          const float wq = c_fq[n][j];
          qp += wq * ir;
          qe += wq * ir * ir * ir;
        }
      ap += (double)c_fq[n][i] * (double)qp;
      ae += (double)c_fq[n][i] * (double)qe;
    }
  *P = ap * kInv4Pi;
  *E = -h * ae * kInv4Pi;
}

__device__ void ort_pe_far32(double a, double b, double c, int n, double* P, double* Ea, double* Eb) {
  const int ne = n + 2;
  const float af = (float)a, bf = (float)b, cf = (float)c;
  const float ap0 = af + 0.5f, am0 = af - 0.5f, bp0 = bf + 0.5f, bm0 = bf - 0.5f;
  double ap = 0.0, aa = 0.0, ab = 0.0;
  for (int sw = -1; sw <= 1; sw += 2) {
    for (int k = 0; k < n; ++k) {
      const float Z = cf + (float)sw * c_fp[n][k];
      const float Z2 = Z * Z;
      float sj = 0.0f;
      for (int j = 0; j < n; ++j) {
        const float q = bf + c_fx[n][j];
        const float bq = q * q + Z2;
        float si = 0.0f;
        for (int i = 0; i < n; ++i) {
          const float pi = af + c_fx[n][i];
          si += c_fw[n][i] * rsqrtf(pi * pi + bq);
        }
        sj += c_fw[n][j] * si;
      }
      ap += (double)c_fq[n][k] * (double)sj;
    }
    for (int k = 0; k < ne; ++k) {
      const float Z = cf + (float)sw * c_fp[ne][k];
      const float Z2 = Z * Z;
      float sa = 0.0f, sb = 0.0f;
      for (int j = 0; j < ne; ++j) {
        const float u = c_fx[ne][j], wu = c_fw[ne][j];
        const float q = bf + u, bq = q * q + Z2;
        const float ra1 = sqrt_approx(ap0 * ap0 + bq), ra0 = sqrt_approx(am0 * am0 + bq);
        sa += wu * __fdividef(-2.0f * af, ra0 * ra1 * (ra0 + ra1));
        const float p = af + u, bp = p * p + Z2;
        const float rb1 = sqrt_approx(bp0 * bp0 + bp), rb0 = sqrt_approx(bm0 * bm0 + bp);
        sb += wu * __fdividef(-2.0f * bf, rb0 * rb1 * (rb0 + rb1));
      }
      aa += (double)c_fq[ne][k] * (double)sa;
      ab += (double)c_fq[ne][k] * (double)sb;
    }
  }
  *P = ap * kInv4Pi;
  *Ea = aa * kInv4Pi;
  *Eb = ab * kInv4Pi;
}

// ---- P and E together at one evaluation point ----
// parallel: P = Ppar(h,s,t), E = dPpar/dh
__device__ void par_pe(double h, double s, double t, double* P, double* E, bool far32 = false) {
  const double gap = fmax(h, fmax(s - 1.0, t - 1.0));
  if (gap <= 1.0) {
    double ap = 0.0, ae = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double wgt = c_cw[i] * c_cw[j];
        const double u = s + (i - 1), v = t + (j - 1);
        ap += wgt * F_par(u, v, h);
        if (h != 0.0) ae += wgt * Fh_par(u, v, h);
      }
    *P = ap * kInv4Pi;
    *E = ae * kInv4Pi;
    return;
  }
  const int n = gl_order_par(gap);
  if (far32) {
    par_pe_far32(h, s, t, n, P, E);
    return;
  }
  double ap = 0.0, ae = 0.0;
  for (int sp = -1; sp <= 1; sp += 2)
    for (int i = 0; i < n; ++i) {
      const double pp = 0.5 * (1.0 + c_glx[n][i]);
      const double wp = 0.5 * c_glw[n][i] * (1.0 - pp);
      const double X = s + sp * pp;
      double qp = 0.0, qe = 0.0;
      for (int sq = -1; sq <= 1; sq += 2)
        for (int j = 0; j < n; ++j) {
          const double qq = 0.5 * (1.0 + c_glx[n][j]);
          const double wq = 0.5 * c_glw[n][j] * (1.0 - qq);
          const double Y = t + sq * qq;
          const double ir = rsqrt(X * X + Y * Y + h * h);
          qp += wq * ir;
          qe += wq * ir * ir * ir;
        }
      ap += wp * qp;
      ae += wp * qe;
    }
  *P = ap * kInv4Pi;
  *E = -h * ae * kInv4Pi;
}

// orthogonal: P = Port(a,b,c), Ea = dPort/da, Eb = dPort/db
__device__ void ort_pe(double a, double b, double c, double* P, double* Ea, double* Eb,
                       bool far32 = false) {
  const double gap = fmax(a - 0.5, fmax(b - 0.5, c - 1.0));
  if (gap <= 1.0) {
    *P = ort_cf(false, a, b, c);
    *Ea = ort_cf(true, a, b, c);
    *Eb = ort_cf(true, b, a, c);
    return;
  }
  // the normal-derivative rules integrate a difference of two potentials;
  // they take two more orders, and 1/r1 - 1/r0 is formed without cancellation
  // as ((a-1/2)^2 - (a+1/2)^2) / (r0 r1 (r0 + r1)) = -2a / (r0 r1 (r0 + r1)).
  const int n = gl_order_ort(gap);
  if (far32) {
    ort_pe_far32(a, b, c, n, P, Ea, Eb);
    return;
  }
  const int ne = n + 2;
  double ap = 0.0, aa = 0.0, ab = 0.0;
  for (int sw = -1; sw <= 1; sw += 2) {
    for (int k = 0; k < n; ++k) {
      const double ww = 0.5 * (1.0 + c_glx[n][k]);
      const double wz = 0.5 * c_glw[n][k] * (1.0 - ww);
      const double Z = c + sw * ww;
      const double Z2 = Z * Z;
      for (int j = 0; j < n; ++j) {
        const double q = b + 0.5 * c_glx[n][j];
        const double bq = q * q + Z2;
        double sp = 0.0;
        for (int i = 0; i < n; ++i) {
          const double pi = a + 0.5 * c_glx[n][i];
          sp += 0.5 * c_glw[n][i] * rsqrt(pi * pi + bq);
        }
        ap += wz * 0.5 * c_glw[n][j] * sp;
      }
    }
    for (int k = 0; k < ne; ++k) {
      const double ww = 0.5 * (1.0 + c_glx[ne][k]);
      const double wz = 0.5 * c_glw[ne][k] * (1.0 - ww);
      const double Z = c + sw * ww;
      const double Z2 = Z * Z;
      for (int j = 0; j < ne; ++j) {
        const double u = 0.5 * c_glx[ne][j];
        const double wu = 0.5 * c_glw[ne][j];
        const double q = b + u, bq = q * q + Z2;          // Ea: q over the test panel
        const double ra1 = sqrt((a + 0.5) * (a + 0.5) + bq), ra0 = sqrt((a - 0.5) * (a - 0.5) + bq);
        aa += wz * wu * (-2.0 * a / (ra0 * ra1 * (ra0 + ra1)));
        const double p = a + u, bp = p * p + Z2;          // Eb: p over the source panel
        const double rb1 = sqrt((b + 0.5) * (b + 0.5) + bp), rb0 = sqrt((b - 0.5) * (b - 0.5) + bp);
        ab += wz * wu * (-2.0 * b / (rb0 * rb1 * (rb0 + rb1)));
      }
    }
  }
  *P = ap * kInv4Pi;
  *Ea = aa * kInv4Pi;
  *Eb = ab * kInv4Pi;
}

struct ToepLaunch {
  double* out[kNumKernels];
  int far32;              // far field with FP32 sums
  int d[6][3];            // extents of the 6 evaluation groups
  int64_t start[7];
};

// Six groups of evaluation points fill the 15 tensors: group a < 3 gives
// P^{aa} and E^{aa} (the same parallel geometry); group 3 + q for the pair
// (a, b) = (x,y), (x,z), (y,z) gives P^{ab}, E^{ab} = dPort/da and
// E^{ba} = dPort/db at the same orthogonal geometry and Toeplitz index.
__global__ void k_toeplitz(ToepLaunch L) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.start[6]) return;
  int gi = 0;
  while (t >= L.start[gi + 1]) ++gi;
  const int64_t q = t - L.start[gi];
  const int dx = L.d[gi][0], dy = L.d[gi][1];
  const int e[3] = {(int)(q % dx), (int)((q / dx) % dy), (int)(q / ((int64_t)dx * dy))};
  if (gi < 3) {
    const int al = gi;
    const int a1 = al == 0 ? 1 : 0, a2 = al == 2 ? 1 : 2;
    if (e[al] <= 1 && e[a1] <= 2 && e[a2] <= 2) return;     // near field: k_toeplitz_near
    double P, E;
    par_pe((double)e[al], (double)e[a1], (double)e[a2], &P, &E, L.far32 != 0);
    L.out[al][q] = P;
    L.out[6 + al][q] = E;
  } else {
    const int pair = gi - 3;
    const int al = pair == 2 ? 1 : 0, be = pair == 0 ? 1 : 2, ga = 3 - al - be;
    if (e[al] <= 1 && e[be] <= 1 && e[ga] <= 2) return;      // near field: k_toeplitz_near
    double P, Ea, Eb;
    ort_pe(e[al] + 0.5, e[be] + 0.5, (double)e[ga], &P, &Ea, &Eb, L.far32 != 0);
    L.out[3 + pair][q] = P;
    L.out[9 + pair][q] = Ea;
    L.out[12 + pair][q] = Eb;
  }
}

// The near-field entries (gap <= 1 voxel: closed-form corner sums in FP64),
// one warp per entry and one lane per corner term.  Blocks 0..53: parallel
// groups, offsets (h, s, t) in {0,1} x {0,1,2}^2; blocks 54..89: orthogonal
// groups, Toeplitz offsets {0,1}^2 x {0,1,2}.
constexpr int kNearBlocks = 3 * 18 + 3 * 12;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_toeplitz_near(ToepLaunch L) {
  const int b = blockIdx.x, lane = threadIdx.x;
  int gi, e[3];
  if (b < 54) {
    gi = b / 18;
    const int r = b % 18, al = gi, a1 = al == 0 ? 1 : 0, a2 = al == 2 ? 1 : 2;
    e[al] = r / 9;
    e[a1] = (r / 3) % 3;
    e[a2] = r % 3;
  } else {
    gi = 3 + (b - 54) / 12;
    const int r = (b - 54) % 12, pair = gi - 3;
    const int al = pair == 2 ? 1 : 0, be = pair == 0 ? 1 : 2, ga = 3 - al - be;
    e[al] = r / 6;
    e[be] = (r / 3) % 2;
    e[ga] = r % 3;
  }
  for (int a = 0; a < 3; ++a)
    if (e[a] >= L.d[gi][a]) return;                  // offset outside this grid's tables
  const int64_t q = (int64_t)e[0] + (int64_t)L.d[gi][0] * (e[1] + (int64_t)L.d[gi][1] * e[2]);
  if (gi < 3) {
    const int al = gi, a1 = al == 0 ? 1 : 0, a2 = al == 2 ? 1 : 2;
    const double h = e[al], s = e[a1], t = e[a2];
    double vp = 0.0, ve = 0.0;
    if (lane < 18) {
      const int m = lane % 9, i = m / 3, j = m % 3;
      const double wgt = c_cw[i] * c_cw[j];
      const double u = s + (i - 1), v = t + (j - 1);
      if (lane < 9) vp = wgt * F_par(u, v, h);
      else if (h != 0.0) ve = wgt * Fh_par(u, v, h);
    }
    vp = warp_sum(vp);
    ve = warp_sum(ve);
    if (lane == 0) {
      L.out[al][q] = vp * kInv4Pi;
      L.out[6 + al][q] = ve * kInv4Pi;
    }
  } else {
    const int pair = gi - 3;
    const int al = pair == 2 ? 1 : 0, be = pair == 0 ? 1 : 2, ga = 3 - al - be;
    const double A = e[al] + 0.5, B = e[be] + 0.5, Cc = e[ga];
    double acc[3] = {0.0, 0.0, 0.0};                 // P, Ea, Eb
    for (int m = lane; m < 36; m += 32) {
      const int comp = m / 12, idx = m % 12;
      const int s1 = (idx & 1) ? 1 : -1, s2 = (idx & 2) ? 1 : -1, j = idx / 4;
      const double wgt = (double)(s1 * s2) * c_cw[j];
      const double w = Cc + (j - 1);
      if (comp == 0) acc[0] += wgt * H_ort(A + 0.5 * s1, B + 0.5 * s2, w);
      else if (comp == 1) acc[1] += wgt * Hp_ort(A + 0.5 * s1, B + 0.5 * s2, w);
      else acc[2] += wgt * Hp_ort(B + 0.5 * s1, A + 0.5 * s2, w);
    }
    for (int c = 0; c < 3; ++c) acc[c] = warp_sum(acc[c]);
    if (lane == 0) {
      L.out[3 + pair][q] = acc[0] * kInv4Pi;
      L.out[9 + pair][q] = acc[1] * kInv4Pi;
      L.out[12 + pair][q] = acc[2] * kInv4Pi;
    }
  }
}

void toeplitz_dims(const Geom& g, int kk, int* d) {
  const int te = ker_test(kk), so = ker_src(kk);
  const int n[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) d[a] = n[a];
  if (te == so) d[te] = n[te] + 1;
}

int build_toeplitz(Handle& h) {
  VC_TRY(ensure_gl_tables());
  ToepLaunch L;
  for (int kk = 0; kk < kNumKernels; ++kk) {
    int* d = h.tdims[kk];
    toeplitz_dims(h.g, kk, d);
    VC_TRY(h.toep[kk].alloc((size_t)d[0] * d[1] * d[2]));
    L.out[kk] = h.toep[kk].p;
  }
  // groups 0..2 share the extents of P^{aa}; groups 3..5 those of P^{ab}
  L.start[0] = 0;
  for (int gi = 0; gi < 6; ++gi) {
    const int* d = h.tdims[gi];
    for (int a = 0; a < 3; ++a) L.d[gi][a] = d[a];
    L.start[gi + 1] = L.start[gi] + (int64_t)d[0] * d[1] * d[2];
  }
  L.far32 = h.far32 ? 1 : 0;
  const int TB = 128;
  const int64_t tot = L.start[6];
  k_toeplitz<<<(unsigned)((tot + TB - 1) / TB), TB, 0, h.stream>>>(L); ::vc::note_launch();
  k_toeplitz_near<<<kNearBlocks, 32, 0, h.stream>>>(L); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

// ---- canonical tensors on an index cube (installation stage) ----
__global__ void k_canonical(int D, double* ppar, double* epar, double* port, double* eort) {
  const int64_t n = (int64_t)D * D * D;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int e0 = (int)(t % D), e1 = (int)((t / D) % D), e2 = (int)(t / ((int64_t)D * D));
  if (ppar || epar) {
    double P, E;
    par_pe((double)e0, (double)e1, (double)e2, &P, &E);
    if (ppar) ppar[t] = P;
    if (epar) epar[t] = E;
  }
  if (port || eort) {
    double P, Ea, Eb;
    ort_pe(e0 + 0.5, e1 + 0.5, (double)e2, &P, &Ea, &Eb);
    if (port) port[t] = P;
    if (eort) eort[t] = Ea;
  }
}

int canonical_tensors(int D, double* ppar, double* epar, double* port, double* eort) {
  VC_TRY(ensure_gl_tables());
  const int64_t n = (int64_t)D * D * D;
  const int TB = 128;
  k_canonical<<<(unsigned)((n + TB - 1) / TB), TB>>>(D, ppar, epar, port, eort); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  VC_CUDA(cudaDeviceSynchronize());
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
    double P, Ev;
    par_pe(fabs(dd[te]), fabs(dd[a1]), fabs(dd[a2]), &P, &Ev);
    v = E ? Ev : P;
  } else {
    const int ga = 3 - te - sr;
    double P, Ea, Eb;
    ort_pe(fabs(dd[te]), fabs(dd[sr]), fabs(dd[ga]), &P, &Ea, &Eb);
    v = E ? Ea : P;
  }
  if (E && dd[te] < 0.0) v = -v;
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
