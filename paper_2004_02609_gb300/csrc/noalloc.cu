// voxcap_matvec_noalloc: the product of voxcap_matvec without any device
// allocation, for callers that must not allocate once they are running.
//
// voxcap_matvec keeps its FFT intermediates in a workspace that the handle
// allocates (and grows) on first use, and its preconditioned form allocates
// one more temporary per call.  This variant takes all of that scratch from
// one fixed array in the library's device image instead, so the call itself
// issues no cudaMalloc / cudaFree.  The array belongs to the library's
// device module: a device holds it from the first call there (which loads
// the module) until the process exits.
#include "internal.h"

namespace vc {

// Maximum scratch of one call: 16 MiB.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with the handle's device current, on every call: the lookup is cheap once
// the library's module is loaded on the device (the first lookup loads it,
// together with the array), and a fresh lookup stays valid after the
// device's context has been torn down and re-created.
static int noalloc_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    set_error(std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") +
              cudaGetErrorString(e));
    return VOXCAP_ERR_CUDA;
  }
  *out = p;
  return VOXCAP_OK;
}

template <typename T>
static int matvec_noalloc_impl(Handle& h, const T* x, T* y, int nrhs, int flags, void* scratch) {
  using C = C_t<T>;
  const bool adj = flags & VOXCAP_MV_ADJOINT;
  if (flags & VOXCAP_MV_RONLY) return precond_apply<T>(h, x, y, nrhs);
  const size_t ws = mvm_workspace_bytes(h, nrhs, sizeof(C));
  size_t need = ws;
  size_t tmp_off = 0;
  if (flags & VOXCAP_MV_PRECOND) {
    tmp_off = (ws + 255) & ~(size_t)255;
    need = tmp_off + sizeof(T) * (size_t)h.pan.N * nrhs;
  }
  VC_CHECK(need <= kNoAllocScratchBytes, VOXCAP_ERR_ARG,
           "voxcap_matvec_noalloc needs " + std::to_string(need) +
               " bytes of scratch for this handle and nrhs, more than its fixed maximum of " +
               std::to_string(kNoAllocScratchBytes) + " bytes; use voxcap_matvec or fewer columns");
  if (flags & VOXCAP_MV_PRECOND) {
    T* t = reinterpret_cast<T*>(static_cast<unsigned char*>(scratch) + tmp_off);
    VC_TRY(mvm<T>(h, x, t, nrhs, adj, nullptr, scratch));
    return precond_apply<T>(h, t, y, nrhs);
  }
  return mvm<T>(h, x, y, nrhs, adj, nullptr, scratch);
}

}  // namespace vc

struct voxcap {
  vc::Handle h;
};

extern "C" int voxcap_matvec_noalloc(voxcap_t* hv, const void* x_dev, void* y_dev, int nrhs,
                                     int dtype, int flags) {
  using namespace vc;
  VC_CHECK(hv != nullptr, VOXCAP_ERR_ARG, "NULL handle");
  VC_CHECK(x_dev && y_dev && x_dev != y_dev, VOXCAP_ERR_ARG, "x and y must be distinct device arrays");
  VC_CHECK(nrhs >= 1, VOXCAP_ERR_ARG, "nrhs must be >= 1");
  VC_CHECK(dtype == VOXCAP_F32 || dtype == VOXCAP_F64, VOXCAP_ERR_ARG, "dtype must be F32 or F64");
  Handle& h = hv->h;
  if (h.pan.N == 0) return VOXCAP_OK;
  int cur = 0;
  VC_CUDA(cudaGetDevice(&cur));
  if (cur != h.device) VC_CUDA(cudaSetDevice(h.device));
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc == VOXCAP_OK) {
    if (dtype == VOXCAP_F32)
      rc = matvec_noalloc_impl<float>(h, (const float*)x_dev, (float*)y_dev, nrhs, flags, scratch);
    else
      rc = matvec_noalloc_impl<double>(h, (const double*)x_dev, (double*)y_dev, nrhs, flags, scratch);
  }
  if (cur != h.device) cudaSetDevice(cur);
  return rc;
}
