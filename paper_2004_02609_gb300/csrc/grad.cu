// Adjoint gradient of the capacitance matrix with respect to the
// permittivities of the material labels.
//
// C_ij = eps0 dv w_i^T rho_j with A rho_j = b_j (Eqs. 4, 8).  Only the
// dielectric diagonal I' (Eq. 7) and the free-charge factors w (eps_r of a
// conductor panel's dielectric side) depend on eps, so for
// L = sum_ij G_ij C_ij and G' = eps0 dv G:
//   dL/d th = sum_j [ (d(W G')_j/d th)^T rho_j - mu_j^T (dA/d th) rho_j ],
//   A^T mu_j = (W G')_j         (one batched adjoint solve, conjugated kernels).
// On a dielectric face f the rows of A and A^T give rho_f = -(M rho)_f / I'_f
// and mu_f = -(M^T mu)_f / I'_f, where M is A without its I' diagonal.  Hence
//   -mu_f rho_f dI'/d eps = -(dI'/d eps / I'^2) (M^T mu)_f (M rho)_f,
//   dI'/d eps_a / I'^2 = -4 eps_b / (eps_a + eps_b)^2,
//   dI'/d eps_b / I'^2 = +4 eps_a / (eps_a + eps_b)^2,
// which stays finite as eps_a -> eps_b, so every face between two dielectric
// voxels contributes, panel or not (the limit of a panel whose I' -> inf).
// (M rho)_f and (M^T mu)_f at every face come from one forward and one
// transposed FP64 product that also write their face-grid fields.
#include <vector>

#include "internal.h"

namespace vc {

__global__ void k_adj_rhs(int64_t N, int m, const int8_t* kind, const int16_t* owner,
                          const double* qscale, const int32_t* struct_of, const double* Gp,
                          double* rhs) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * m) return;
  const int j = (int)(t / N);
  const int64_t p = t % N;
  double v = 0.0;
  if (kind[p] == 0) {
    const int s = struct_of[p];
    v = qscale[p] * Gp[((int64_t)s * m + owner[p]) * m + j];
  }
  rhs[t] = v;
}

// per-face I' terms
__global__ void k_grad_faces(Geom g, int S, int m, const int32_t* __restrict__ labels,
                             const int32_t* __restrict__ cid, const double* __restrict__ eps,
                             const double* __restrict__ ffwd, const double* __restrict__ fadj,
                             double* __restrict__ grad) {
  const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
  const int64_t box = g.box();
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)S * 3 * box) return;
  const int s = (int)(t / (3 * box));
  const int o = (int)((t / box) % 3);
  const int64_t f = t % box;
  const int i = (int)(f % g.Lx), j = (int)((f / g.Lx) % g.Ly), k = (int)(f / ((int64_t)g.Lx * g.Ly));
  const int n[3] = {g.nx, g.ny, g.nz};
  int c[3] = {i, j, k};
  // is (i,j,k) a face of orientation o?
  for (int a = 0; a < 3; ++a)
    if (c[a] > n[a] - (a == o ? 0 : 1)) return;
  const int32_t* lab = labels + (int64_t)s * nvox;
  int ca[3] = {i, j, k};
  ca[o] -= 1;
  const int la = ca[o] >= 0 ? lab[(int64_t)ca[0] + (int64_t)g.nx * (ca[1] + (int64_t)g.ny * ca[2])] : -1;
  const int lb = c[o] < n[o] ? lab[(int64_t)c[0] + (int64_t)g.nx * (c[1] + (int64_t)g.ny * c[2])] : -1;
  if ((la >= 0 && cid[la] >= 0) || (lb >= 0 && cid[lb] >= 0)) return;
  if (la < 0 && lb < 0) return;
  const double ea = la >= 0 ? eps[la] : 1.0, eb = lb >= 0 ? eps[lb] : 1.0;
  const double sum = ea + eb;
  double F = 0.0;
  for (int q = 0; q < m; ++q) {
    const int64_t b = (int64_t)s * m + q;
    const int64_t idx = (b * 3 + o) * box + f;
    F += ffwd[idx] * fadj[idx];
  }
  if (F == 0.0) return;
  if (la >= 0) atomicAdd(&grad[la], 4.0 * eb / (sum * sum) * F);
  if (lb >= 0) atomicAdd(&grad[lb], -4.0 * ea / (sum * sum) * F);
}

// free-charge factor terms: w_{i,p} = eps of the dielectric side of conductor panel p
__global__ void k_grad_w(int64_t N, int m, const int8_t* kind, const int16_t* owner,
                         const int32_t* la, const int32_t* lb, const int32_t* cid,
                         const int32_t* struct_of, const double* Gp, const double* rho,
                         double* grad) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N || kind[p] != 0) return;
  const int a = la[p], b = lb[p];
  const int other = (a >= 0 && cid[a] >= 0) ? b : a;
  if (other < 0) return;                      // vacuum outside the grid: fixed
  const int s = struct_of[p], i = owner[p];
  double v = 0.0;
  for (int j = 0; j < m; ++j) v += Gp[((int64_t)s * m + i) * m + j] * rho[(int64_t)j * N + p];
  atomicAdd(&grad[other], v);
}

int capacitance_grad(Handle& h, const double* dLdC, double tol, double* grad_host, voxcap_stats* st) {
  const int m = h.pan.m_max, S = h.pan.S;
  const int64_t N = h.pan.N;
  const Geom& g = h.g;
  const double eps0 = 8.8541878128e-12;
  std::vector<double> Gp((size_t)S * m * m);
  for (size_t q = 0; q < Gp.size(); ++q) Gp[q] = eps0 * h.dv * dLdC[q];
  DBuf<double> Gd, rhs, mu, y, ff, fa, gd;
  VC_TRY(Gd.alloc(Gp.size()));
  VC_TRY(rhs.alloc((size_t)N * m));
  VC_TRY(mu.alloc((size_t)N * m));
  VC_TRY(y.alloc((size_t)N * m));
  const size_t nf = (size_t)S * m * 3 * g.box();
  VC_TRY(ff.alloc(nf));
  VC_TRY(fa.alloc(nf));
  VC_TRY(gd.alloc((size_t)h.nlab));
  VC_CUDA(cudaMemcpyAsync(Gd.p, Gp.data(), sizeof(double) * Gp.size(), cudaMemcpyHostToDevice, h.stream));
  VC_CUDA(cudaMemsetAsync(gd.p, 0, sizeof(double) * h.nlab, h.stream));
  VC_CUDA(cudaMemsetAsync(ff.p, 0, sizeof(double) * nf, h.stream));
  VC_CUDA(cudaMemsetAsync(fa.p, 0, sizeof(double) * nf, h.stream));
  const int TB = 256;
  k_adj_rhs<<<(unsigned)((N * m + TB - 1) / TB), TB, 0, h.stream>>>(
      N, m, h.pan.kind.p, h.pan.owner.p, h.pan.qscale.p, h.pan.struct_of.p, Gd.p, rhs.p);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  int rc = solve(h, rhs.p, m, tol, mu.p, st, true);
  if (rc != VOXCAP_OK && rc != VOXCAP_ERR_NOT_CONVERGED) return rc;
  VC_TRY(mvm<double>(h, h.rho.p, y.p, m, false, ff.p));
  VC_TRY(mvm<double>(h, mu.p, y.p, m, true, fa.p));
  const int64_t nfaces = (int64_t)S * 3 * g.box();
  k_grad_faces<<<(unsigned)((nfaces + TB - 1) / TB), TB, 0, h.stream>>>(
      g, S, m, h.labels.p, h.cid_d.p, h.eps_d.p, ff.p, fa.p, gd.p);
  ::vc::note_launch();
  k_grad_w<<<(unsigned)((N + TB - 1) / TB), TB, 0, h.stream>>>(
      N, m, h.pan.kind.p, h.pan.owner.p, h.pan.la.p, h.pan.lb.p, h.cid_d.p, h.pan.struct_of.p, Gd.p,
      h.rho.p, gd.p);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  VC_CUDA(cudaMemcpyAsync(grad_host, gd.p, sizeof(double) * h.nlab, cudaMemcpyDeviceToHost, h.stream));
  VC_CUDA(cudaStreamSynchronize(h.stream));
  for (int l = 0; l < h.nlab; ++l)
    if (h.cid[l] >= 0) grad_host[l] = 0.0;
  return rc;
}

}  // namespace vc
