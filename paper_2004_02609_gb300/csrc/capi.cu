// extern "C" entry points declared in include/voxcap.h.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace vc {
const char* last_error();
void toeplitz_dims(const Geom& g, int kk, int* d);
int build_toeplitz_tucker(Handle& h, const voxcap_tucker& tk);
int canonical_tensors(int D, double* ppar, double* epar, double* port, double* eort);
}

struct voxcap {
  vc::Handle h;
};

using namespace vc;

extern "C" {

void voxcap_default_opts(voxcap_opts* o) {
  if (!o) return;
  o->precision = VOXCAP_FP32_REFINE;
  o->restart = 35;
  o->inner_tol = 1e-4;
  o->max_iters = 2000;
  o->max_sweeps = 20;
  o->nv[0] = o->nv[1] = o->nv[2] = 10;
  o->precond = VOXCAP_PRECOND_BDD;
  o->pad_mode = 0;
  o->entries = VOXCAP_ENTRIES_AUTO;
  o->tucker = nullptr;
  o->fast_refine = 0;
}

const char* voxcap_last_error(void) { return vc::last_error(); }

static int setup_impl(const int32_t* labels, int nx, int ny, int nz, int n_struct,
                      const int32_t* conductor_id, const double* eps_r, int n_labels,
                      double voxel_size_m, const voxcap_opts* opts, void* cuda_stream,
                      voxcap_t** out) {
  VC_CHECK(out != nullptr, VOXCAP_ERR_ARG, "out is NULL");
  *out = nullptr;
  VC_CHECK(labels && conductor_id && eps_r, VOXCAP_ERR_ARG, "NULL input array");
  VC_CHECK(nx > 0 && ny > 0 && nz > 0 && n_struct > 0 && n_labels > 0, VOXCAP_ERR_ARG,
           "grid sizes, n_struct and n_labels must be positive");
  VC_CHECK(voxel_size_m > 0.0, VOXCAP_ERR_ARG, "voxel_size_m must be positive");
  VC_CHECK((int64_t)nx * ny * nz < (int64_t)1 << 31, VOXCAP_ERR_ARG, "grid too large");
  for (int l = 0; l < n_labels; ++l) {
    VC_CHECK(conductor_id[l] >= -1, VOXCAP_ERR_ARG, "conductor_id must be >= -1");
    VC_CHECK(conductor_id[l] >= 0 || (eps_r[l] > 0.0 && eps_r[l] < 1e300), VOXCAP_ERR_ARG,
             "eps_r must be positive and finite for dielectric labels");
  }
  voxcap* v = new (std::nothrow) voxcap;
  VC_CHECK(v != nullptr, VOXCAP_ERR_OOM, "host allocation failed");
  Handle& h = v->h;
  auto fail = [&](int rc) { delete v; return rc; };
  int rc;
  VC_CUDA(cudaGetDevice(&h.device));
  h.stream = (cudaStream_t)cuda_stream;
  set_alloc_stream(h.stream);
  if (opts) h.opts = *opts; else voxcap_default_opts(&h.opts);
  if (h.opts.restart < 1) h.opts.restart = 35;
  VC_CHECK(h.opts.restart <= kMaxRestart, VOXCAP_ERR_ARG,
           "restart must be at most " + std::to_string(kMaxRestart));
  if (h.opts.max_iters < 1) h.opts.max_iters = 2000;
  VC_CHECK(h.opts.entries >= VOXCAP_ENTRIES_AUTO && h.opts.entries <= VOXCAP_ENTRIES_FAR32, VOXCAP_ERR_ARG,
           "entries must be one of VOXCAP_ENTRIES_*");
  // permittivity contrast (vacuum outside the grid included): on dielectric
  // rows I' + E' nearly cancel at high contrast and amplify entry errors by
  // about the contrast, so FP32 far-field sums are only automatic up to 1e4
  double emin = 1.0, emax = 1.0;
  for (int l = 0; l < n_labels; ++l)
    if (conductor_id[l] < 0) {
      emin = std::min(emin, eps_r[l]);
      emax = std::max(emax, eps_r[l]);
    }
  h.far32 = h.opts.entries == VOXCAP_ENTRIES_FAR32 ||
            (h.opts.entries == VOXCAP_ENTRIES_AUTO && h.opts.precision == VOXCAP_FP32_REFINE &&
             emax <= 1e4 * emin);
  h.dv = voxel_size_m;
  h.nlab = n_labels;
  h.cid.assign(conductor_id, conductor_id + n_labels);
  h.eps.assign(eps_r, eps_r + n_labels);
  Geom& g = h.g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.Lx = nx + 1; g.Ly = ny + 1; g.Lz = nz + 1;
  h.pan.S = n_struct;
  const size_t nl = (size_t)n_struct * nx * ny * nz;
  if ((rc = h.labels.alloc(nl))) return fail(rc);
  if ((rc = h.cid_d.alloc(n_labels))) return fail(rc);
  if ((rc = h.eps_d.alloc(n_labels))) return fail(rc);
  cudaPointerAttributes attr;
  cudaError_t ae = cudaPointerGetAttributes(&attr, labels);
  (void)cudaGetLastError();
  const bool on_dev = ae == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  if (cudaMemcpyAsync(h.labels.p, labels, nl * sizeof(int32_t),
                      on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h.stream) != cudaSuccess ||
      cudaMemcpyAsync(h.cid_d.p, conductor_id, n_labels * sizeof(int32_t), cudaMemcpyHostToDevice,
                      h.stream) != cudaSuccess ||
      cudaMemcpyAsync(h.eps_d.p, eps_r, n_labels * sizeof(double), cudaMemcpyHostToDevice, h.stream) !=
          cudaSuccess) {
    set_error(std::string("copy of the inputs failed: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(VOXCAP_ERR_CUDA);
  }
  // phase wall times (the stream is drained at each mark)
  auto tp = std::chrono::steady_clock::now();
  auto mark = [&](int i) {
    cudaStreamSynchronize(h.stream);
    const auto t = std::chrono::steady_clock::now();
    h.setup_s[i] = std::chrono::duration<double>(t - tp).count();
    tp = t;
  };
  if ((rc = build_fft_plans(h))) return fail(rc);
  mark(0);
  if ((rc = build_panels(h))) return fail(rc);
  mark(1);
  if (h.opts.tucker) {
    if ((rc = build_toeplitz_tucker(h, *h.opts.tucker))) return fail(rc);
  } else if ((rc = build_toeplitz(h))) {
    return fail(rc);
  }
  h.opts.tucker = nullptr;        // the caller's factors are not retained
  mark(2);
  if ((rc = build_spectra(h))) return fail(rc);
  mark(3);
  if ((rc = build_precond(h))) return fail(rc);
  mark(4);
  if ((rc = tune_products(h))) return fail(rc);
  mark(5);
  *out = v;
  return VOXCAP_OK;
}

int voxcap_setup(const int32_t* labels, int nx, int ny, int nz, int n_struct,
                 const int32_t* conductor_id, const double* eps_r, int n_labels,
                 double voxel_size_m, const voxcap_opts* opts, void* cuda_stream,
                 voxcap_t** out) {
  try {
    return setup_impl(labels, nx, ny, nz, n_struct, conductor_id, eps_r, n_labels, voxel_size_m,
                      opts, cuda_stream, out);
  } catch (...) {
    set_error("unexpected host exception in voxcap_setup");
    return VOXCAP_ERR_ARG;
  }
}

void voxcap_destroy(voxcap_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->h.stream);
  delete h;
}

int voxcap_num_panels(const voxcap_t* hv, int s, int64_t* n_cond, int64_t* n_diel, int* n_conductors,
                      int64_t* n_total, int64_t* offset) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  const Panels& P = hv->h.pan;
  VC_CHECK(s >= 0 && s < P.S, VOXCAP_ERR_ARG, "structure index out of range");
  if (n_cond) *n_cond = P.nc[s];
  if (n_diel) *n_diel = P.nd[s];
  if (n_conductors) *n_conductors = P.m[s];
  if (n_total) *n_total = P.N;
  if (offset) *offset = P.off[s];
  return VOXCAP_OK;
}

int voxcap_panel_map(const voxcap_t* hv, int s, int8_t* orient, int32_t* face_idx, int8_t* kind,
                     int16_t* owner, double* idiag, double* qscale) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  const Handle& h = hv->h;
  const Panels& P = h.pan;
  VC_CHECK(s >= 0 && s < P.S, VOXCAP_ERR_ARG, "structure index out of range");
  const int64_t o = P.off[s], n = P.nc[s] + P.nd[s];
  if (n == 0) return VOXCAP_OK;
  if (orient) VC_CUDA(cudaMemcpy(orient, P.orient.p + o, n, cudaMemcpyDeviceToHost));
  if (face_idx) VC_CUDA(cudaMemcpy(face_idx, P.face.p + o, n * 4, cudaMemcpyDeviceToHost));
  if (kind) VC_CUDA(cudaMemcpy(kind, P.kind.p + o, n, cudaMemcpyDeviceToHost));
  if (owner) VC_CUDA(cudaMemcpy(owner, P.owner.p + o, n * 2, cudaMemcpyDeviceToHost));
  if (idiag) VC_CUDA(cudaMemcpy(idiag, P.idiag.p + o, n * 8, cudaMemcpyDeviceToHost));
  if (qscale) VC_CUDA(cudaMemcpy(qscale, P.qscale.p + o, n * 8, cudaMemcpyDeviceToHost));
  return VOXCAP_OK;
}

int voxcap_matvec(voxcap_t* hv, const void* x_dev, void* y_dev, int nrhs, int dtype, int flags) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  set_alloc_stream(hv->h.stream);
  VC_CHECK(x_dev && y_dev && x_dev != y_dev, VOXCAP_ERR_ARG, "x and y must be distinct device arrays");
  VC_CHECK(nrhs >= 1, VOXCAP_ERR_ARG, "nrhs must be >= 1");
  VC_CHECK(dtype == VOXCAP_F32 || dtype == VOXCAP_F64, VOXCAP_ERR_ARG, "dtype must be F32 or F64");
  Handle& h = hv->h;
  const bool adj = flags & VOXCAP_MV_ADJOINT;
  const int64_t N = h.pan.N;
  if (N == 0) return VOXCAP_OK;
  if (flags & VOXCAP_MV_RONLY) {
    if (dtype == VOXCAP_F32) return precond_apply<float>(h, (const float*)x_dev, (float*)y_dev, nrhs);
    return precond_apply<double>(h, (const double*)x_dev, (double*)y_dev, nrhs);
  }
  if (dtype == VOXCAP_F32) {
    if (flags & VOXCAP_MV_PRECOND) {
      DBuf<float> t;
      VC_TRY(t.alloc((size_t)N * nrhs));
      VC_TRY(mvm<float>(h, (const float*)x_dev, t.p, nrhs, adj, nullptr));
      VC_TRY(precond_apply<float>(h, t.p, (float*)y_dev, nrhs));
      VC_CUDA(cudaStreamSynchronize(h.stream));
      return VOXCAP_OK;
    }
    return mvm<float>(h, (const float*)x_dev, (float*)y_dev, nrhs, adj, nullptr);
  }
  if (flags & VOXCAP_MV_PRECOND) {
    DBuf<double> t;
    VC_TRY(t.alloc((size_t)N * nrhs));
    VC_TRY(mvm<double>(h, (const double*)x_dev, t.p, nrhs, adj, nullptr));
    VC_TRY(precond_apply<double>(h, t.p, (double*)y_dev, nrhs));
    VC_CUDA(cudaStreamSynchronize(h.stream));
    return VOXCAP_OK;
  }
  return mvm<double>(h, (const double*)x_dev, (double*)y_dev, nrhs, adj, nullptr);
}

int voxcap_solve(voxcap_t* hv, const double* B_dev, int nrhs, double tol, double* X_dev,
                 voxcap_stats* st) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  set_alloc_stream(hv->h.stream);
  VC_CHECK(B_dev && X_dev && nrhs >= 1, VOXCAP_ERR_ARG, "bad solve arguments");
  VC_CHECK(tol > 0.0 && tol < 1.0, VOXCAP_ERR_ARG, "tol must be in (0, 1)");
  return solve(hv->h, B_dev, nrhs, tol, X_dev, st, false);
}

int voxcap_capacitance(voxcap_t* hv, double tol, double* C_host, double* rho_dev, voxcap_stats* st) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  set_alloc_stream(hv->h.stream);
  VC_CHECK(C_host != nullptr, VOXCAP_ERR_ARG, "C_host is NULL");
  VC_CHECK(tol > 0.0 && tol < 1.0, VOXCAP_ERR_ARG, "tol must be in (0, 1)");
  return capacitance(hv->h, tol, C_host, rho_dev, st);
}

int voxcap_capacitance_columns(voxcap_t* hv, double tol, int j0, int j1, double* C_host, voxcap_stats* st) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  set_alloc_stream(hv->h.stream);
  VC_CHECK(C_host != nullptr, VOXCAP_ERR_ARG, "C_host is NULL");
  VC_CHECK(tol > 0.0 && tol < 1.0, VOXCAP_ERR_ARG, "tol must be in (0, 1)");
  VC_CHECK(hv->h.pan.m_max > 0, VOXCAP_ERR_NO_CONDUCTOR, "no conductor in the material table");
  VC_CHECK(j0 >= 0 && j1 > j0 && j1 <= hv->h.pan.m_max, VOXCAP_ERR_ARG, "conductor range outside [0, m)");
  return capacitance_cols(hv->h, tol, j0, j1, C_host, nullptr, st);
}

int voxcap_capacitance_grad(voxcap_t* hv, const double* dL_dC_host, double tol, double* grad_host,
                            voxcap_stats* st) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  set_alloc_stream(hv->h.stream);
  VC_CHECK(dL_dC_host && grad_host, VOXCAP_ERR_ARG, "NULL array");
  VC_CHECK(hv->h.have_rho, VOXCAP_ERR_ARG, "call voxcap_capacitance first");
  VC_CHECK(tol > 0.0 && tol < 1.0, VOXCAP_ERR_ARG, "tol must be in (0, 1)");
  return capacitance_grad(hv->h, dL_dC_host, tol, grad_host, st);
}

int voxcap_update_eps(voxcap_t* hv, const double* eps_r) {
  VC_CHECK(hv != nullptr && eps_r != nullptr, VOXCAP_ERR_ARG, "NULL argument");
  set_alloc_stream(hv->h.stream);
  Handle& h = hv->h;
  for (int l = 0; l < h.nlab; ++l)
    VC_CHECK(h.cid[l] >= 0 || (eps_r[l] > 0.0 && eps_r[l] < 1e300), VOXCAP_ERR_ARG,
             "eps_r must be positive and finite for dielectric labels");
  h.eps.assign(eps_r, eps_r + h.nlab);
  VC_CUDA(cudaMemcpyAsync(h.eps_d.p, eps_r, sizeof(double) * h.nlab, cudaMemcpyHostToDevice, h.stream));
  h.gm.reset();                   // the restart-cycle graph points into the rebuilt tables
  VC_TRY(build_panels(h));
  VC_TRY(build_precond(h));
  h.have_rho = false;
  return VOXCAP_OK;
}

int voxcap_entries(int n, const int32_t* kind, const int32_t* test_orient, const int32_t* src_orient,
                   const double* d, double* out) {
  VC_CHECK(n >= 0, VOXCAP_ERR_ARG, "n must be >= 0");
  if (n == 0) return VOXCAP_OK;
  VC_CHECK(kind && test_orient && src_orient && d && out, VOXCAP_ERR_ARG, "NULL array");
  return entries_eval(n, kind, test_orient, src_orient, d, out, nullptr);
}

int voxcap_canonical_tensors(int D, double* ppar, double* epar, double* port, double* eort) {
  VC_CHECK(D > 0 && (int64_t)D * D * D < ((int64_t)1 << 34), VOXCAP_ERR_ARG, "bad cube size");
  return canonical_tensors(D, ppar, epar, port, eort);
}

int64_t voxcap_launch_count(void) { return vc::launch_count(); }

int voxcap_set_product_tiles(voxcap_t* hv, int z_order, int z_tile_log2, int y_fwd_log2, int y_inv_log2,
                             int* choice_out) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  Handle& h = hv->h;
  VC_CHECK(z_order >= -2 && z_order <= 1, VOXCAP_ERR_ARG, "z_order must be -2, -1, 0 or 1");
  if (z_order >= 0)
    VC_CHECK(z_tile_log2 >= 0 && z_tile_log2 <= 4 && y_fwd_log2 >= -1 && y_fwd_log2 <= 4 &&
                 y_inv_log2 >= -1 && y_inv_log2 <= 4,
             VOXCAP_ERR_ARG, "tile widths out of range");
  set_alloc_stream(h.stream);
  if (z_order == -2) {
    // query only
  } else if (z_order < 0) {
    VC_TRY(retune_products(h));
  } else {
    h.path = 0;                       // a forced variant is one of the generic passes
    h.zvar = z_order < h.nzvar ? z_order : 0;
    h.ztx = z_tile_log2;
    h.ytx[0] = y_fwd_log2;
    h.ytx[1] = y_inv_log2;
  }
  if (choice_out) {
    choice_out[0] = h.zvar;
    choice_out[1] = h.ztx;
    choice_out[2] = h.ytx[0];
    choice_out[3] = h.ytx[1];
  }
  return VOXCAP_OK;
}

int voxcap_setup_times(const voxcap_t* hv, double* seconds) {
  VC_CHECK(hv != nullptr && seconds != nullptr, VOXCAP_ERR_ARG, "NULL handle or output");
  for (int i = 0; i < 6; ++i) seconds[i] = hv->h.setup_s[i];
  return VOXCAP_OK;
}

int voxcap_set_product_path(voxcap_t* hv, int path, int* path_out) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  VC_CHECK(path >= -2 && path <= 15 && (path <= 1 || (path & 1)), VOXCAP_ERR_ARG,
           "path must be -2, -1, 0, 1 or 1 plus variant bits 2, 4, 8");
  Handle& h = hv->h;
  set_alloc_stream(h.stream);
  if (path == -2) {
    // query only
  } else if (path < 0) {
    VC_TRY(retune_products(h));
  } else {
    h.path = path & 1;
    h.zfvar = (path >> 1) & 1;
    h.yvar[0] = (path >> 2) & 1;
    h.yvar[1] = (path >> 3) & 1;
  }
  if (path_out) *path_out = h.path == 1 ? 1 | (h.zfvar << 1) | (h.yvar[0] << 2) | (h.yvar[1] << 3) : h.path;
  return VOXCAP_OK;
}

int voxcap_fft_length(const voxcap_t* hv, int* mx, int* my, int* mz) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  if (mx) *mx = hv->h.g.Mx;
  if (my) *my = hv->h.g.My;
  if (mz) *mz = hv->h.g.Mz;
  return VOXCAP_OK;
}

int voxcap_toeplitz(const voxcap_t* hv, int t, double* out_host, int* dims) {
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  VC_CHECK(t >= 0 && t < kNumKernels, VOXCAP_ERR_ARG, "tensor index out of range");
  const Handle& h = hv->h;
  const int* d = h.tdims[t];
  if (dims) { dims[0] = d[0]; dims[1] = d[1]; dims[2] = d[2]; }
  if (out_host)
    VC_CUDA(cudaMemcpy(out_host, h.toep[t].p, sizeof(double) * (size_t)d[0] * d[1] * d[2],
                       cudaMemcpyDeviceToHost));
  return VOXCAP_OK;
}

}  // extern "C"
