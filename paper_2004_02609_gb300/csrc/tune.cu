// Set-up-time autotuning of the product: the radix order of the z pass's
// transform (largest radix <= 9 last, or smallest last) and its tile width
// (8 or 16 columns), then the tile widths of the inverse and forward y passes
// (4, 8 or the default), then the compiled-plan passes where the padded
// lengths have one, are timed on the handle's own FP32 products, all
// conductor columns at once, and the fastest is kept.  The choice is cached
// per device, grid and batch, so later set-ups of the same shape reuse it.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>

#include "fast.cuh"
#include "internal.h"

namespace vc {

namespace {
std::mutex g_tune_mu;
std::map<std::array<int, 8>, std::array<int, 8>> g_tune;
}  // namespace

static int tune(Handle& h, bool use_cache) {
  const int64_t N = h.pan.N;
  if (N == 0) return VOXCAP_OK;
  VC_TRY(h.zqueue.alloc(1));       // before any product: none may allocate inside a captured graph
  const int nrhs = std::max(1, h.pan.m_max);
  const Geom& g = h.g;
  const std::array<int, 8> key = {h.device, g.Mx, g.My, g.Mz, g.nx, g.ny, g.nz, h.pan.S * nrhs};
  if (use_cache) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      h.zvar = it->second[0];
      h.ztx = it->second[1];
      h.ytx[0] = it->second[2];
      h.ytx[1] = it->second[3];
      h.path = it->second[4];
      h.yvar[0] = it->second[5];
      h.yvar[1] = it->second[6];
      h.zfvar = it->second[7];
      return VOXCAP_OK;
    }
  }
  DBuf<float> x, y;
  VC_TRY(x.alloc((size_t)N * nrhs));
  VC_TRY(y.alloc((size_t)N * nrhs));
  VC_CUDA(cudaMemsetAsync(x.p, 0, sizeof(float) * (size_t)N * nrhs, h.stream));
  VC_TRY(mvm_prepare(h, nrhs, sizeof(float2)));
  cudaEvent_t e0, e1;
  VC_CUDA(cudaEventCreate(&e0));
  VC_CUDA(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } guard{e0, e1};
  // times 3 products of the current choice (after one untimed); < 0 if it cannot launch
  auto time_products = [&](float* ms) -> int {
    if (mvm<float>(h, x.p, y.p, nrhs, false, nullptr) != VOXCAP_OK) {
      (void)cudaGetLastError();
      *ms = -1.0f;
      return VOXCAP_OK;
    }
    VC_CUDA(cudaEventRecord(e0, h.stream));
    for (int r = 0; r < 3; ++r) VC_TRY(mvm<float>(h, x.p, y.p, nrhs, false, nullptr));
    VC_CUDA(cudaEventRecord(e1, h.stream));
    VC_CUDA(cudaEventSynchronize(e1));
    VC_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return VOXCAP_OK;
  };
  h.ytx[0] = h.ytx[1] = -1;
  h.path = 0;
  h.yvar[0] = h.yvar[1] = 0;
  h.zfvar = 0;
  float best_ms = 1e30f;
  int best_v = 0, best_tx = -1;
  for (int v = 0; v < h.nzvar; ++v)
    for (int tx : {4, 3}) {
      h.zvar = v;
      h.ztx = tx;
      float ms;
      VC_TRY(time_products(&ms));
      if (ms >= 0.0f && ms < best_ms) {
        best_ms = ms;
        best_v = v;
        best_tx = tx;
      }
    }
  VC_CHECK(best_ms < 1e30f, VOXCAP_ERR_UNSUPPORTED, "no z-pass variant fits this grid");
  h.zvar = best_v;
  h.ztx = best_tx;
  // then the tile widths of the inverse and the forward y passes (-1: the default)
  for (int which : {1, 0}) {
    int best_y = -1;
    for (int t : {3, 2}) {
      h.ytx[which] = t;
      float ms;
      VC_TRY(time_products(&ms));
      if (ms >= 0.0f && ms < best_ms) {
        best_ms = ms;
        best_y = t;
      }
    }
    h.ytx[which] = best_y;
  }
  // then the compiled-plan passes, where the lengths have a plan, in every
  // combination of their variant switches (the persistent z pass, the
  // persistent forward and inverse y passes)
  if (fast_plan_ok(h.pf[1]) || fast_z_ok(h) || fast_x_ok(h)) {
    const bool ypipe = fast_plan_ok(h.pf[1]);
    const bool zpipe = fast_z_ok(h) && h.pzf[0].radix[0] == 16;
    int best_bits = -1;
    for (int bits = 0; bits < 8; ++bits) {
      if (((bits & 1) && !zpipe) || ((bits & 6) && !ypipe)) continue;
      h.path = 1;
      h.zfvar = bits & 1;
      h.yvar[0] = (bits >> 1) & 1;
      h.yvar[1] = (bits >> 2) & 1;
      float ms;
      VC_TRY(time_products(&ms));
      if (ms >= 0.0f && ms < best_ms) {
        best_ms = ms;
        best_bits = bits;
      }
    }
    const int bb = best_bits > 0 ? best_bits : 0;
    h.path = best_bits >= 0 ? 1 : 0;
    h.zfvar = bb & 1;
    h.yvar[0] = (bb >> 1) & 1;
    h.yvar[1] = (bb >> 2) & 1;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {h.zvar, h.ztx, h.ytx[0], h.ytx[1], h.path, h.yvar[0], h.yvar[1], h.zfvar};
  return VOXCAP_OK;
}

int tune_products(Handle& h) { return tune(h, true); }
int retune_products(Handle& h) { return tune(h, false); }

}  // namespace vc
