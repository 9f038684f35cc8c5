// Internal state of a voxcap handle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace vc {

// Device allocations come from the device's stream-ordered memory pool on
// the stream of the calling handle (set on entry to every API call); the pool
// keeps freed memory for reuse, so building and solving repeatedly does not
// go back to cudaMalloc / cudaFree.
void set_alloc_stream(cudaStream_t s);
cudaStream_t alloc_stream();

// A device allocation owned by the handle.
template <typename T> struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  int alloc(size_t count);
  void release();
  ~DBuf() { release(); }
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
};

template <typename T> int DBuf<T>::alloc(size_t count) {
  if (count <= n && p) return VOXCAP_OK;
  release();
  if (count == 0) return VOXCAP_OK;
  st = alloc_stream();
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), st);
  if (e != cudaSuccess) {
    p = nullptr;
    (void)cudaGetLastError();
    set_error("device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    return VOXCAP_ERR_OOM;
  }
  n = count;
  return VOXCAP_OK;
}
template <typename T> void DBuf<T>::release() {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
  n = 0;
}

// Grid geometry shared by all structures of a handle.
struct Geom {
  int nx, ny, nz;      // voxels
  int Lx, Ly, Lz;      // common face box (N+1 per axis)
  int Mx, My, Mz;      // padded FFT lengths (>= 2N+1, even)
  int Hx;              // Mx/2 + 1
  int Oy, Oz;          // My/2 + 1, Mz/2 + 1 (octant extents of the spectra)
  __host__ __device__ int64_t box() const { return (int64_t)Lx * Ly * Lz; }
};

// The 15 kernel tensors: 0..5 P xx,yy,zz,xy,xz,yz ; 6..14 E xx,yy,zz,xy,xz,yz,yx,zx,zy
constexpr int kNumKernels = 15;
// test / source orientation of each kernel tensor
__host__ __device__ __forceinline__ int ker_test(int kk) {
  switch (kk) {
    case 0: case 3: case 4: case 6: case 9: case 10: return 0;
    case 1: case 5: case 7: case 11: case 12: return 1;
    default: return 2;
  }
}
__host__ __device__ __forceinline__ int ker_src(int kk) {
  switch (kk) {
    case 0: case 6: case 12: case 13: return 0;
    case 1: case 3: case 7: case 9: case 14: return 1;
    default: return 2;
  }
}

struct Panels {
  int S = 0;                      // structures
  int64_t N = 0;                  // total panels
  std::vector<int64_t> off, nc, nd;   // per structure
  std::vector<int> m;             // conductors per structure
  int m_max = 0;
  DBuf<int8_t> orient, kind;
  DBuf<int32_t> face;
  DBuf<int16_t> owner;
  DBuf<double> idiag, qscale;     // I' (Eq. 7), free-charge factor
  DBuf<float> idiag_f;
  DBuf<int32_t> la, lb;           // labels of the two sides (-1 outside)
  DBuf<int32_t> fmap;             // [S][3][Lz][Ly][Lx] -> global panel index or -1
  DBuf<int32_t> struct_of;        // [N] structure of each panel
  // panels by face row: the panels of kind k on row (o, z, y) of structure s
  // are [rstart[q], rstart[q + 1]) with q = (2 s + k) R + (o Lz + z) Ly + y,
  // R = 3 Lz Ly (canonical order makes every row one contiguous run), and
  // px[p] is the position of panel p along its row
  DBuf<int32_t> rstart;
  DBuf<int32_t> px;
};

// Pinned host ints the device writes directly (mapped), e.g. the per-step
// active flags of GMRES that the host polls.
struct HostMap {
  int* h = nullptr;
  int* d = nullptr;
  size_t n = 0;
  int ensure(size_t count) {
    if (count <= n && h) return VOXCAP_OK;
    release();
    if (cudaHostAlloc(reinterpret_cast<void**>(&h), count * sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
      h = nullptr;
      (void)cudaGetLastError();
      set_error("mapped host allocation failed");
      return VOXCAP_ERR_OOM;
    }
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), h, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      release();
      set_error("mapped host pointer unavailable");
      return VOXCAP_ERR_CUDA;
    }
    n = count;
    for (size_t i = 0; i < n; ++i) h[i] = 0;
    return VOXCAP_OK;
  }
  void release() {
    if (h) cudaFreeHost(h);
    h = nullptr;
    d = nullptr;
    n = 0;
  }
  ~HostMap() { release(); }
  HostMap() = default;
  HostMap(const HostMap&) = delete;
  HostMap& operator=(const HostMap&) = delete;
};

struct Precond {
  int kind = VOXCAP_PRECOND_BDD;
  int nv[3] = {10, 10, 10};
  int nbx = 0, nby = 0, nbz = 0;
  int64_t nboxes = 0;             // (per structure) * S
  int64_t nblocks = 0;            // non-empty boxes
  int64_t nunique = 0;
  int max_n = 0;
  DBuf<int32_t> blk_off;          // [nblocks+1] offsets into blk_idx
  DBuf<int32_t> blk_idx;          // panel indices, canonical order inside a block
  DBuf<int32_t> blk_uid;          // [nblocks] unique-block id
  DBuf<int64_t> uoff;             // [nunique+1] offsets (elements) of inverse matrices
  DBuf<double> inv_d;             // unique inverses, row-major n x n each
  DBuf<float> inv_f;
  DBuf<double> dscale_d;          // per-panel diagonal factor for rows outside blocks (0 inside)
  DBuf<float> dscale_f;
};

// The instantiated graph of one GMRES restart cycle (a device-side while
// loop over Arnoldi steps), kept per handle and rebuilt when its key (shape,
// precision, workspace addresses, product variant) changes.
struct GmresGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uintptr_t key[10] = {0};
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    for (auto& k : key) k = 0;
  }
  ~GmresGraph() { reset(); }
  GmresGraph() = default;
  GmresGraph(const GmresGraph&) = delete;
  GmresGraph& operator=(const GmresGraph&) = delete;
};

constexpr int kMaxRestart = 512;   // longest GMRES restart cycle (Arnoldi basis of kMaxRestart + 1 vectors)
constexpr int kSpecBlk = 8;      // kx columns per block of the blocked FP32 spectra

struct Handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  voxcap_opts opts;
  // the operator is only FP32-accurate (FP32 far-field entries): its spectra
  // are transformed in FP32 too and the FP64 copy is their widening
  bool far32 = false;
  double dv = 1.0;
  int nlab = 0;
  std::vector<int32_t> cid;
  std::vector<double> eps;
  DBuf<int32_t> labels;           // [S][nz][ny][nx]
  DBuf<int32_t> cid_d;
  DBuf<double> eps_d;
  Geom g;
  Panels pan;
  Precond pre;
  // FFT plans; their stage twiddles and the half-voxel phases live in one
  // device table uploaded with a single copy
  DBuf<char> plan_tab;
  Plan1D<double2> pd[3];
  Plan1D<float2> pf[3];
  // the same transforms with the radix order reversed: the inverse z
  // transform of the products starts with the radix the forward one ends
  // with, so the two meet in registers
  Plan1D<double2> pdr[3];
  Plan1D<float2> pfr[3];
  // z pass: forward/reversed plans of up to two radix orders (0: largest
  // radix <= 9 last, 1: smallest radix last) and the tuned choice
  int nzvar = 1;
  Plan1D<double2> pzd[2], pzdr[2];
  Plan1D<float2> pzf[2], pzfr[2];
  int zvar = 0;                   // radix order of the z pass
  int ztx = -1;                   // log2 of its tile width, -1: heuristic
  int ytx[2] = {-1, -1};          // log2 of the forward / inverse y passes' tile widths (FP32)
  // FP32 product kernels: 0 generic passes, 1 compiled-plan passes where the
  // padded lengths have a compiled plan (fast_*.cu), -1 not chosen yet
  int path = -1;
  int yvar[2] = {0, 0};           // variants of the compiled forward / inverse y passes (tile width)
  int zfvar = 0;                  // variant of the compiled z pass (0 one tile per CTA, 1 persistent)
  DBuf<int> zqueue;               // tile counter of the persistent z pass (allocated at set-up)
  const double2* phd[3] = {nullptr, nullptr, nullptr};   // exp(+i pi k / M) per axis, k in [0, M)
  const float2* phf[3] = {nullptr, nullptr, nullptr};
  // Toeplitz tensors (FP64) and spectra
  int tdims[kNumKernels][3];
  DBuf<double> toep[kNumKernels];
  DBuf<double> spec_d;            // [15][Oz][Oy][Hx] real, scaled by 1/(Mx My Mz)
  DBuf<float> spec_f;
  // the same FP32 spectra in blocks of kSpecBlk consecutive kx for the
  // compiled z pass: [Oy][ceil(Hx / kSpecBlk)][Oz][15][kSpecBlk] (zero past
  // Hx), so that the spectra of a tile of columns are one contiguous block
  DBuf<float> spec_fb;
  // MVM workspace
  int ws_batch = 0;
  DBuf<char> ws;                  // raw workspace
  // solver workspace and results
  DBuf<double> rho;               // last capacitance charges N x m_max
  DBuf<double> rhs;               // last capacitance RHS
  bool have_rho = false;
  DBuf<char> solver_ws;
  GmresGraph gm;                  // restart-cycle graph (declared after the buffers it points into)
  double setup_s[6] = {0, 0, 0, 0, 0, 0};   // wall seconds of the set-up phases (voxcap_setup_times)
  HostMap act_map;                // GMRES: [2][nrhs] active flags per step parity, then the
                                  // cycle-end read-back of iteration counts and flags [2][nrhs]
};

// ---- per-precision views of the handle's plans, phases and spectra
template <typename T> inline const Plan1D<C_t<T>>& plan_of(const Handle& h, int a);
template <> inline const Plan1D<float2>& plan_of<float>(const Handle& h, int a) { return h.pf[a]; }
template <> inline const Plan1D<double2>& plan_of<double>(const Handle& h, int a) { return h.pd[a]; }
template <typename T> inline const Plan1D<C_t<T>>& plan_rev_of(const Handle& h, int a);
template <> inline const Plan1D<float2>& plan_rev_of<float>(const Handle& h, int a) { return h.pfr[a]; }
template <> inline const Plan1D<double2>& plan_rev_of<double>(const Handle& h, int a) { return h.pdr[a]; }
template <typename T> inline const C_t<T>* phase_of(const Handle& h, int a);
template <> inline const float2* phase_of<float>(const Handle& h, int a) { return h.phf[a]; }
template <> inline const double2* phase_of<double>(const Handle& h, int a) { return h.phd[a]; }
template <typename T> inline const T* spec_of(const Handle& h);
template <> inline const float* spec_of<float>(const Handle& h) { return h.spec_f.p; }
template <> inline const double* spec_of<double>(const Handle& h) { return h.spec_d.p; }

// opt a kernel in to `bytes` of dynamic shared memory
template <typename K> inline int set_smem(K kernel, size_t bytes) {
  VC_CHECK(bytes <= 227 * 1024, VOXCAP_ERR_UNSUPPORTED, "FFT tile does not fit in shared memory");
  VC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return VOXCAP_OK;
}

// The z pass of a product (z transforms, spectral multiply-accumulate,
// inverse z transforms) over B batch items of the y/z-pass buffer, in place;
// radix order `var` and tile width 2^tx_sh (tx_sh < 0: the handle's choice).
template <typename T, bool ADJ>
int zmac_launch(const Handle& h, C_t<T>* data, int B, cudaStream_t st, int var = -1, int tx_sh = -1);
// Time the z-pass variants on this handle's own FP32 products and keep the
// fastest (cached per grid shape and batch).
int tune_products(Handle& h);
int retune_products(Handle& h);   // the same, ignoring (and replacing) the cached choice

// ---- module entry points (host side) ----
int build_fft_plans(Handle& h);
int build_panels(Handle& h);
int build_toeplitz(Handle& h);
int build_spectra(Handle& h);
int build_precond(Handle& h);
// y = A x (or A^T x) for `nrhs` columns of the handle's N panels.
// field_out (optional, double only): face-grid fields [nrhs][3][box] written
// for every face (E-part for forward, full adjoint output for adjoint).
// workspace: caller-provided scratch of at least mvm_workspace_bytes(); when
// NULL the handle's own workspace is used (allocated or grown on demand).
template <typename T>
int mvm(Handle& h, const T* x, T* y, int nrhs, bool adjoint, T* field_out,
        void* workspace = nullptr);
size_t mvm_workspace_bytes(const Handle& h, int nrhs, size_t complex_bytes);
// constant tables and workspace of the product for nrhs columns
int mvm_prepare(Handle& h, int nrhs, size_t complex_bytes);
template <typename T>
int precond_apply(Handle& h, const T* r, T* z, int nrhs);
int solve(Handle& h, const double* B, int nrhs, double tol, double* X, voxcap_stats* st,
          bool adjoint);
int capacitance(Handle& h, double tol, double* C_host, double* rho_dev, voxcap_stats* st);
int capacitance_cols(Handle& h, double tol, int j0, int j1, double* C_host, double* rho_dev, voxcap_stats* st);
int capacitance_grad(Handle& h, const double* dLdC, double tol, double* grad_host,
                     voxcap_stats* st);
// entries evaluated on arbitrary (kind, orientations, centre difference)
int entries_eval(int n, const int32_t* kind, const int32_t* to, const int32_t* so,
                 const double* d, double* out, cudaStream_t st);

}  // namespace vc
