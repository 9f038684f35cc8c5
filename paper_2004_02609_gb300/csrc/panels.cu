// Voxel labels -> conductor / dielectric panels (Sec. II.A-B; Eqs. 3-4, 7).
//
// One thread per face of the three face grids classifies the face from the
// voxels on its two sides; a device-wide exclusive scan over the flags in
// canonical order (conductor rows first, then orientation x<y<z, then face
// index) gives every panel its row; a second pass writes the panel arrays
// and the face -> panel maps that the FFT scatter / gather passes read.
#include "internal.h"

namespace vc {

struct FaceGrid {
  int F[3][3];          // dims of the face grid of each orientation
  int64_t cnt[3];       // faces per orientation
  int64_t start[3];     // offset of orientation o in a [3][faces] sequence
  int64_t total;
};

static FaceGrid face_grid(const Geom& g) {
  FaceGrid fg;
  int64_t s = 0;
  for (int o = 0; o < 3; ++o) {
    int d[3] = {g.nx, g.ny, g.nz};
    d[o] += 1;
    for (int a = 0; a < 3; ++a) fg.F[o][a] = d[a];
    fg.cnt[o] = (int64_t)d[0] * d[1] * d[2];
    fg.start[o] = s;
    s += fg.cnt[o];
  }
  fg.total = s;
  return fg;
}

struct FaceInfo {
  int cls;        // 0 none, 1 conductor panel, 2 dielectric panel, -1 short, -2 bad label
  int la, lb;     // labels of the two sides (-1 outside)
  int owner;
  double ea, eb;
};

__device__ __forceinline__ FaceInfo classify(const int32_t* __restrict__ lab, int nx, int ny, int nz,
                                             const int32_t* __restrict__ cid,
                                             const double* __restrict__ eps, int nlab, int o,
                                             int i, int j, int k) {
  FaceInfo fi;
  int ia[3] = {i, j, k};
  int ib[3] = {i, j, k};
  ia[o] -= 1;   // -axis side voxel
  const int dims[3] = {nx, ny, nz};
  fi.la = -1; fi.lb = -1;
  if (ia[o] >= 0) fi.la = lab[(int64_t)ia[0] + (int64_t)nx * (ia[1] + (int64_t)ny * ia[2])];
  if (ib[o] < dims[o]) fi.lb = lab[(int64_t)ib[0] + (int64_t)nx * (ib[1] + (int64_t)ny * ib[2])];
  if (fi.la >= nlab || fi.lb >= nlab || fi.la < -1 || fi.lb < -1 ||
      (ia[o] >= 0 && fi.la < 0) || (ib[o] < dims[o] && fi.lb < 0)) {
    fi.cls = -2; return fi;
  }
  int ca = fi.la >= 0 ? cid[fi.la] : -1;
  int cb = fi.lb >= 0 ? cid[fi.lb] : -1;
  fi.ea = fi.la >= 0 ? eps[fi.la] : 1.0;
  fi.eb = fi.lb >= 0 ? eps[fi.lb] : 1.0;
  fi.owner = -1;
  if (ca >= 0 && cb >= 0) {
    fi.cls = (ca == cb) ? 0 : -1;
  } else if (ca >= 0 || cb >= 0) {
    fi.cls = 1;
    fi.owner = ca >= 0 ? ca : cb;
  } else {
    fi.cls = (fi.ea != fi.eb) ? 2 : 0;
  }
  return fi;
}

__global__ void k_classify(const int32_t* __restrict__ lab, int nx, int ny, int nz,
                           const int32_t* __restrict__ cid, const double* __restrict__ eps,
                           int nlab, FaceGrid fg, int32_t* __restrict__ flags,
                           int* __restrict__ err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= fg.total) return;
  int o = (t >= fg.start[2]) ? 2 : (t >= fg.start[1] ? 1 : 0);
  int64_t f = t - fg.start[o];
  int Fx = fg.F[o][0], Fy = fg.F[o][1];
  int i = (int)(f % Fx), j = (int)((f / Fx) % Fy), k = (int)(f / ((int64_t)Fx * Fy));
  FaceInfo fi = classify(lab, nx, ny, nz, cid, eps, nlab, o, i, j, k);
  if (fi.cls < 0) {
    atomicMax(err, fi.cls == -1 ? 1 : 2);
    fi.cls = 0;
  }
  flags[t] = (fi.cls == 1);
  flags[fg.total + t] = (fi.cls == 2);
}

__global__ void k_scatter_panels(const int32_t* __restrict__ lab, int nx, int ny, int nz,
                                 const int32_t* __restrict__ cid, const double* __restrict__ eps,
                                 int nlab, FaceGrid fg, const int32_t* __restrict__ pos,
                                 int64_t off, int s, Geom g,
                                 int8_t* orient, int32_t* face, int8_t* kind, int16_t* owner,
                                 double* idiag, float* idiag_f, double* qscale, int32_t* la,
                                 int32_t* lb, int32_t* fmap, int32_t* struct_of) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= fg.total) return;
  int o = (t >= fg.start[2]) ? 2 : (t >= fg.start[1] ? 1 : 0);
  int64_t f = t - fg.start[o];
  int Fx = fg.F[o][0], Fy = fg.F[o][1];
  int i = (int)(f % Fx), j = (int)((f / Fx) % Fy), k = (int)(f / ((int64_t)Fx * Fy));
  FaceInfo fi = classify(lab, nx, ny, nz, cid, eps, nlab, o, i, j, k);
  if (fi.cls != 1 && fi.cls != 2) return;
  int64_t p = off + (fi.cls == 1 ? pos[t] : pos[fg.total + t]);
  orient[p] = (int8_t)o;
  face[p] = (int32_t)f;
  kind[p] = (int8_t)(fi.cls - 1);
  owner[p] = (int16_t)fi.owner;
  la[p] = fi.la;
  lb[p] = fi.lb;
  struct_of[p] = s;
  if (fi.cls == 1) {
    idiag[p] = 0.0;
    idiag_f[p] = 0.0f;
    qscale[p] = (fi.owner == (fi.la >= 0 ? cid[fi.la] : -2)) ? fi.eb : fi.ea;
  } else {
    double I = (fi.ea + fi.eb) / (2.0 * (fi.ea - fi.eb));
    idiag[p] = I;
    idiag_f[p] = (float)I;
    qscale[p] = 0.0;
  }
  fmap[(((int64_t)s * 3 + o) * g.Lz + k) * ((int64_t)g.Ly * g.Lx) + (int64_t)j * g.Lx + i] = (int32_t)p;
}

// panels per face row, by structure and kind (see Panels::rstart)
__global__ void k_row_count(int64_t N, const int8_t* __restrict__ orient, const int32_t* __restrict__ face,
                            const int8_t* __restrict__ kind, const int32_t* __restrict__ struct_of, Geom g,
                            int32_t* __restrict__ cnt, int32_t* __restrict__ px) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int o = orient[p];
  const int Fx = o == 0 ? g.nx + 1 : g.nx, Fy = o == 1 ? g.ny + 1 : g.ny;
  const int64_t f = face[p];
  const int i = (int)(f % Fx), j = (int)((f / Fx) % Fy), k = (int)(f / ((int64_t)Fx * Fy));
  const int64_t R = 3 * (int64_t)g.Lz * g.Ly;
  const int64_t q = (2 * (int64_t)struct_of[p] + kind[p]) * R + ((int64_t)o * g.Lz + k) * g.Ly + j;
  atomicAdd(cnt + q, 1);
  px[p] = i;
}

int build_panels(Handle& h) {
  Geom& g = h.g;
  Panels& P = h.pan;
  const int S = P.S;
  FaceGrid fg = face_grid(g);
  const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;
  DBuf<int32_t> flags, tmp;
  DBuf<int> err;
  VC_TRY(flags.alloc((size_t)(2 * fg.total)));
  VC_TRY(tmp.alloc((size_t)scan_tmp_elems(2 * fg.total)));
  VC_TRY(err.alloc(1));
  // pass 1: counts per structure
  std::vector<int64_t> cnt_c(S), cnt_d(S);
  const int TB = 256;
  unsigned nblk = (unsigned)((fg.total + TB - 1) / TB);
  int64_t ntot = 0;
  for (int s = 0; s < S; ++s) {
    VC_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), h.stream));
    k_classify<<<nblk, TB, 0, h.stream>>>(h.labels.p + s * nvox, g.nx, g.ny, g.nz, h.cid_d.p,
                                         h.eps_d.p, h.nlab, fg, flags.p, err.p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
    int e = 0;
    VC_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    VC_CUDA(cudaStreamSynchronize(h.stream));
    VC_CHECK(e != 1, VOXCAP_ERR_SHORT,
             "structure " + std::to_string(s) + ": two different conductors share a face");
    VC_CHECK(e != 2, VOXCAP_ERR_ARG,
             "structure " + std::to_string(s) + ": voxel label outside [0, n_labels)");
    int64_t total = 0;
    // count conductor flags separately: scan the whole [2][faces] sequence and
    // read the running sum at the kind boundary
    VC_TRY(exclusive_scan_i32(flags.p, 2 * fg.total, tmp.p, &total, h.stream));
    int32_t at_split = 0;
    VC_CUDA(cudaMemcpyAsync(&at_split, flags.p + fg.total, sizeof(int32_t), cudaMemcpyDeviceToHost,
                            h.stream));
    VC_CUDA(cudaStreamSynchronize(h.stream));
    cnt_c[s] = at_split;
    cnt_d[s] = total - at_split;
    ntot += total;
  }
  VC_CHECK(ntot < (int64_t)INT32_MAX, VOXCAP_ERR_ARG, "more than 2^31 panels");
  P.N = ntot;
  P.off.assign(S, 0);
  P.nc = cnt_c;
  P.nd = cnt_d;
  int64_t o = 0;
  for (int s = 0; s < S; ++s) { P.off[s] = o; o += cnt_c[s] + cnt_d[s]; }
  size_t N = (size_t)std::max<int64_t>(ntot, 1);
  VC_TRY(P.orient.alloc(N)); VC_TRY(P.kind.alloc(N)); VC_TRY(P.face.alloc(N));
  VC_TRY(P.owner.alloc(N)); VC_TRY(P.idiag.alloc(N)); VC_TRY(P.qscale.alloc(N));
  VC_TRY(P.idiag_f.alloc(N)); VC_TRY(P.la.alloc(N)); VC_TRY(P.lb.alloc(N));
  VC_TRY(P.struct_of.alloc(N));
  VC_TRY(P.fmap.alloc((size_t)S * 3 * g.box()));
  VC_CUDA(cudaMemsetAsync(P.fmap.p, 0xFF, sizeof(int32_t) * (size_t)S * 3 * g.box(), h.stream));
  // pass 2: positions + scatter.  The dielectric positions of the scan are
  // relative to the start of the sequence, i.e. already offset by the number
  // of conductor panels, as the canonical order requires.
  for (int s = 0; s < S; ++s) {
    int32_t* dummy_err = err.p;
    k_classify<<<nblk, TB, 0, h.stream>>>(h.labels.p + s * nvox, g.nx, g.ny, g.nz, h.cid_d.p,
                                         h.eps_d.p, h.nlab, fg, flags.p, dummy_err); ::vc::note_launch();
    VC_TRY(exclusive_scan_i32(flags.p, 2 * fg.total, tmp.p, nullptr, h.stream));
    k_scatter_panels<<<nblk, TB, 0, h.stream>>>(
        h.labels.p + s * nvox, g.nx, g.ny, g.nz, h.cid_d.p, h.eps_d.p, h.nlab, fg, flags.p,
        P.off[s], s, g, P.orient.p, P.face.p, P.kind.p, P.owner.p, P.idiag.p, P.idiag_f.p,
        P.qscale.p, P.la.p, P.lb.p, P.fmap.p, P.struct_of.p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  // face rows: counts by (structure, kind, row), then an exclusive scan; in
  // canonical order the scan of a row is the index of its first panel
  {
    const int64_t nrows = 2 * (int64_t)S * 3 * g.Lz * g.Ly;
    VC_CHECK(nrows < (int64_t)INT32_MAX, VOXCAP_ERR_ARG, "too many face rows");
    VC_TRY(P.rstart.alloc((size_t)nrows + 1));
    VC_TRY(P.px.alloc(N));
    DBuf<int32_t> stmp;
    VC_TRY(stmp.alloc((size_t)scan_tmp_elems(nrows + 1)));
    VC_CUDA(cudaMemsetAsync(P.rstart.p, 0, sizeof(int32_t) * (size_t)(nrows + 1), h.stream));
    if (ntot > 0) {
      k_row_count<<<(unsigned)((ntot + TB - 1) / TB), TB, 0, h.stream>>>(ntot, P.orient.p, P.face.p, P.kind.p,
                                                                       P.struct_of.p, g, P.rstart.p, P.px.p);
      ::vc::note_launch();
      VC_CUDA(cudaGetLastError());
    }
    int64_t tot = 0;
    VC_TRY(exclusive_scan_i32(P.rstart.p, nrows + 1, stmp.p, &tot, h.stream));
    VC_CHECK(tot == ntot, VOXCAP_ERR_CUDA, "face-row counts do not add up to the panel count");
  }
  // conductors per structure: largest owner + 1 over the structure's labels
  P.m.assign(S, 0);
  int mc = 0;
  for (int l = 0; l < h.nlab; ++l) mc = std::max(mc, h.cid[l] + 1);
  for (int s = 0; s < S; ++s) P.m[s] = mc;
  P.m_max = mc;
  VC_CUDA(cudaStreamSynchronize(h.stream));
  return VOXCAP_OK;
}

}  // namespace vc
