// Block-diagonal-diagonal preconditioner (Eq. 14, Sec. II.D) and the
// comparison variants of Sec. III.A.
//
// The bounding box is split into small boxes of nv[0] x nv[1] x nv[2] voxels.
// A face at index i along its own normal axis belongs to box
// min(i / nv, n_boxes - 1) (the far boundary faces join the last box) and to
// box j / nv along the other axes.  For the paper's preconditioner (BDD) the
// block of a box holds the conductor panels it owns, with entries P' read
// from the FP64 Toeplitz tensors; its inverse preconditions those conductor
// rows, and dielectric rows are scaled by 1/I'.  Boxes whose panel pattern
// (orientations and face offsets from the box corner) is identical have
// identical blocks, so only one inverse per distinct pattern is stored
// (Sec. II.D point (ii)).  BD uses all panels of a box (dielectric rows with
// E' + I'), DIAG uses 1/A_kk and NONE the identity.  Inverses of blocks up to
// 224 panels are computed in FP32 by one CTA each (a preconditioner only
// steers GMRES); larger blocks by a multi-CTA FP64 Gauss-Jordan.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace vc {

struct BoxGeom {
  int n[3], nv[3], nb[3];
  int64_t nbox;      // boxes per structure
  int Lx, Ly, Lz;
};

// Panels selected for blocks: BDD -> conductor panels only; BD -> all.
__device__ __forceinline__ bool selected(int kind, int mode) {
  return mode == VOXCAP_PRECOND_BD || kind == 0;
}

// face-index range [lo, hi) of box coordinate bc along axis a for orientation o
__device__ __forceinline__ void box_range(const BoxGeom& bg, int o, int a, int bc, int* lo, int* hi) {
  *lo = bc * bg.nv[a];
  int h = (bc + 1) * bg.nv[a];
  if (a == o) {
    if (bc == bg.nb[a] - 1) h = bg.n[a] + 1;
  } else if (h > bg.n[a]) {
    h = bg.n[a];
  }
  *hi = h;
}

// Walk the faces of one box in canonical order (orientation, face index);
// `fn(p, o, i, j, k)` is called for every selected panel, in order, by the
// whole block cooperatively; returns the count.  Two phases: count, then fill.
template <bool FILL>
__device__ int walk_box(const BoxGeom& bg, int s, int64_t box, const int32_t* __restrict__ fmap,
                        const int8_t* __restrict__ kind, int mode, int32_t* __restrict__ out) {
  __shared__ int warp_tot[32];
  __shared__ int base_sh;
  const int bx = (int)(box % bg.nb[0]);
  const int by = (int)((box / bg.nb[0]) % bg.nb[1]);
  const int bz = (int)(box / ((int64_t)bg.nb[0] * bg.nb[1]));
  const int bcs[3] = {bx, by, bz};
  if (threadIdx.x == 0) base_sh = 0;
  __syncthreads();
  for (int o = 0; o < 3; ++o) {
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) box_range(bg, o, a, bcs[a], &lo[a], &hi[a]);
    const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
    const int cnt = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
    const int32_t* fm = fmap + ((int64_t)s * 3 + o) * ((int64_t)bg.Lz * bg.Ly * bg.Lx);
    for (int c0 = 0; c0 < cnt; c0 += blockDim.x) {
      const int c = c0 + threadIdx.x;
      int p = -1;
      if (c < cnt) {
        const int i = lo[0] + c % ex, j = lo[1] + (c / ex) % ey, k = lo[2] + c / (ex * ey);
        p = fm[((int64_t)k * bg.Ly + j) * bg.Lx + i];
        if (p >= 0 && !selected(kind[p], mode)) p = -1;
      }
      const int flag = p >= 0;
      // block exclusive scan of flags
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      int v = flag;
      for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
      }
      if (lane == 31) warp_tot[wid] = v;
      __syncthreads();
      if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
          int t = __shfl_up_sync(0xffffffffu, w, d);
          if (lane >= d) w += t;
        }
        warp_tot[lane] = w;
      }
      __syncthreads();
      const int excl = v - flag + (wid > 0 ? warp_tot[wid - 1] : 0);
      const int tot = warp_tot[(blockDim.x >> 5) - 1];
      if (FILL && flag) out[base_sh + excl] = p;
      __syncthreads();
      if (threadIdx.x == 0) base_sh += tot;
      __syncthreads();
    }
  }
  return base_sh;
}

__global__ void k_box_count(BoxGeom bg, const int32_t* fmap, const int8_t* kind, int mode,
                            int32_t* counts) {
  const int64_t gb = blockIdx.x;          // s * nbox + box
  const int s = (int)(gb / bg.nbox);
  const int64_t box = gb % bg.nbox;
  int n = walk_box<false>(bg, s, box, fmap, kind, mode, nullptr);
  if (threadIdx.x == 0) counts[gb] = n;
}

__global__ void k_box_fill(BoxGeom bg, const int32_t* fmap, const int8_t* kind, int mode,
                           const int32_t* offs, int32_t* idx) {
  const int64_t gb = blockIdx.x;
  const int s = (int)(gb / bg.nbox);
  const int64_t box = gb % bg.nbox;
  walk_box<true>(bg, s, box, fmap, kind, mode, idx + offs[gb]);
}

// local pattern key of panel p in box gb: orientation, offsets from the box corner, kind
__device__ __forceinline__ uint64_t pat_key(const BoxGeom& bg, int64_t gb, int p,
                                            const int8_t* orient, const int32_t* face,
                                            const int8_t* kind, const double* idiag, int mode) {
  const int64_t box = gb % bg.nbox;
  const int bx = (int)(box % bg.nb[0]);
  const int by = (int)((box / bg.nb[0]) % bg.nb[1]);
  const int bz = (int)(box / ((int64_t)bg.nb[0] * bg.nb[1]));
  const int o = orient[p];
  int F[3] = {bg.n[0], bg.n[1], bg.n[2]};
  F[o] += 1;
  const int f = face[p];
  const int i = f % F[0], j = (f / F[0]) % F[1], k = f / (F[0] * F[1]);
  uint64_t key = (uint64_t)o;
  key = key * 4099u + (uint64_t)(i - bx * bg.nv[0]);
  key = key * 4099u + (uint64_t)(j - by * bg.nv[1]);
  key = key * 4099u + (uint64_t)(k - bz * bg.nv[2]);
  key = key * 3u + (uint64_t)kind[p];
  if (mode == VOXCAP_PRECOND_BD && kind[p] == 1) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(idiag[p]);
    key ^= bits * 0x9E3779B97F4A7C15ull;
  }
  return key;
}

// hash of a box's pattern: the sum of its mixed panel keys (order-free; the
// representative search below compares patterns exactly).  One warp per box.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_box_hash(BoxGeom bg, int64_t nboxes, const int32_t* offs, const int32_t* idx,
                           const int8_t* orient, const int32_t* face, const int8_t* kind,
                           const double* idiag, int mode, uint64_t* hash) {
  const int64_t gb = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gb >= nboxes) return;                          // whole warps leave together
  uint64_t hsh = 0;
  for (int q = offs[gb] + lane; q < offs[gb + 1]; q += 32)
    hsh += mix64(pat_key(bg, gb, idx[q], orient, face, kind, idiag, mode));
  for (int o = 16; o > 0; o >>= 1) hsh += __shfl_down_sync(0xffffffffu, hsh, o);
  if (lane == 0) hash[gb] = hsh + (uint64_t)(offs[gb + 1] - offs[gb]);
}

// representative = lowest-index box with the same pattern (exact comparison)
__global__ void k_box_rep(BoxGeom bg, int64_t nboxes, const int32_t* offs, const int32_t* idx,
                          const int8_t* orient, const int32_t* face, const int8_t* kind,
                          const double* idiag, int mode, const uint64_t* hash, int32_t* rep,
                          int32_t* is_rep) {
  int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gb >= nboxes) return;
  const int n = offs[gb + 1] - offs[gb];
  int r = (int)gb;
  if (n > 0) {
    for (int64_t c = 0; c < gb; ++c) {
      if (hash[c] != hash[gb] || offs[c + 1] - offs[c] != n) continue;
      bool same = true;
      for (int q = 0; q < n && same; ++q)
        same = pat_key(bg, c, idx[offs[c] + q], orient, face, kind, idiag, mode) ==
               pat_key(bg, gb, idx[offs[gb] + q], orient, face, kind, idiag, mode);
      if (same) { r = (int)c; break; }
    }
  }
  rep[gb] = r;
  is_rep[gb] = (n > 0 && r == (int)gb) ? 1 : 0;
}

__global__ void k_box_uid(int64_t nboxes, const int32_t* rep, const int32_t* rep_scan,
                          const int32_t* offs, int32_t* uid) {
  int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gb >= nboxes) return;
  uid[gb] = (offs[gb + 1] > offs[gb]) ? rep_scan[rep[gb]] : -1;
}

// ---- entry of A between two panels from the Toeplitz tensors ----
struct ToepTabs {
  const double* T[kNumKernels];
  int d[kNumKernels][3];
  int n[3];
};

__device__ __forceinline__ int tidx_p(int a, int b) {
  if (a == b) return a;
  int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}
__device__ __forceinline__ int tidx_e(int a, int b) {
  if (a == b) return 6 + a;
  if (a == 0) return b == 1 ? 9 : 10;
  if (a == 1) return b == 2 ? 11 : 12;
  return b == 0 ? 13 : 14;
}

// A_kl for test panel (ot, it[]) and source (os, is[]) (face-grid coordinates)
__device__ double a_entry(const ToepTabs& tt, bool E, int ot, const int* it, int os, const int* is) {
  int te = ot, so = os;
  int d[3] = {it[0] - is[0], it[1] - is[1], it[2] - is[2]};
  int kk;
  if (!E) {
    // P is symmetric: P^{ba}(d) = P^{ab}(-d); tables exist for a <= b
    kk = tidx_p(te, so);
    if (te > so) {
      int t = te; te = so; so = t;
      d[0] = -d[0]; d[1] = -d[1]; d[2] = -d[2];
    }
  } else {
    kk = tidx_e(te, so);
  }
  double sg = 1.0;
  int e[3];
  for (int a = 0; a < 3; ++a) {
    const int v = d[a];
    if (te == so) {
      e[a] = v < 0 ? -v : v;
      if (E && a == te && v < 0) sg = -sg;
    } else if (a == te) {
      e[a] = v >= 1 ? v - 1 : -v;
      if (E && v < 1) sg = -sg;
    } else if (a == so) {
      e[a] = v >= 0 ? v : -v - 1;
    } else {
      e[a] = v < 0 ? -v : v;
    }
  }
  const int* dd = tt.d[kk];
  return sg * tt.T[kk][(int64_t)e[0] + (int64_t)dd[0] * (e[1] + (int64_t)dd[1] * e[2])];
}

__device__ __forceinline__ void face_coords(const int* n, int o, int f, int* c) {
  int F[3] = {n[0], n[1], n[2]};
  F[o] += 1;
  c[0] = f % F[0];
  c[1] = (f / F[0]) % F[1];
  c[2] = f / (F[0] * F[1]);
}

// assemble [A_B | I] (n x 2n, row-major) for one unique block
__global__ void k_assemble(ToepTabs tt, const int32_t* urep, const int32_t* offs, const int32_t* idx,
                           const int64_t* aoff, const int8_t* orient, const int32_t* face,
                           const int8_t* kind, const double* idiag, double* aug) {
  const int u = blockIdx.x;
  const int gb = urep[u];
  const int q0 = offs[gb];
  const int n = offs[gb + 1] - q0;
  double* Mx = aug + aoff[u];
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    const int pk = idx[q0 + i], pl = idx[q0 + j];
    int ck[3], cl[3];
    face_coords(tt.n, orient[pk], face[pk], ck);
    face_coords(tt.n, orient[pl], face[pl], cl);
    const bool E = kind[pk] == 1;
    double v = a_entry(tt, E, orient[pk], ck, orient[pl], cl);
    if (E && i == j) v += idiag[pk];
    Mx[(int64_t)i * 2 * n + j] = v;
    Mx[(int64_t)i * 2 * n + n + j] = (i == j) ? 1.0 : 0.0;
  }
}

// Inverse of one unique block of n <= 224 panels, held in shared memory by
// one CTA of 32 warps (FP32; the preconditioner only steers GMRES, the
// solution's accuracy comes from the residuals).  In-place Gauss-Jordan
// with pivot bookkeeping: step k takes as pivot the unused row p_k with the
// largest |S[p][k]|, scales that row and eliminates column k from every
// other row; column k, now a unit vector, stores column p_k of the
// inverse-to-be, and A^-1[q_i][p_j] = S[i][j] at the end (q = p^-1).
// Blocked by panels K of 16 columns: the steps of a panel touch only its
// columns (warp c < 16 owns panel column c, so the owner of the next column
// finds its pivot without a barrier; one barrier per step publishes the
// pivot column), then the panel's transformation T_K x = x (rows P_K zeroed)
// + S[:, K] x[P_K] is applied to every other column as one rank-16 update
// by all 32 warps.
constexpr int kGJTileMax = 224;
constexpr int kGJPanel = 16;                     // = warps per CTA

__global__ void __launch_bounds__(1024, 1)
k_block_inverse(ToepTabs tt, const int32_t* __restrict__ urep, const int32_t* __restrict__ offs,
                const int32_t* __restrict__ idx, const int64_t* __restrict__ uoff,
                const int8_t* __restrict__ orient, const int32_t* __restrict__ face,
                const int8_t* __restrict__ kind, const double* __restrict__ idiag,
                double* __restrict__ inv_d, float* __restrict__ inv_f, int* __restrict__ status) {
  extern __shared__ float gj_sm[];
  __shared__ float colb[2][kGJTileMax];
  __shared__ int perm[kGJTileMax], qinv[kGJTileMax];
  __shared__ unsigned char used[kGJTileMax];
  __shared__ int prow[2];
  __shared__ float pinv[2];
  __shared__ int pan_rows[kGJPanel];
  __shared__ int fail;
  const int u = blockIdx.x;
  const int gb = urep[u];
  const int q0 = offs[gb];
  const int n = offs[gb + 1] - q0;
  if (n > kGJTileMax || n == 0) return;              // larger blocks take the multi-CTA path
  const int ld = n | 1;
  float* S = gj_sm;                                  // [n][ld]
  float* Bp = gj_sm + (size_t)n * ld;                // [kGJPanel][ld]: rows P_K before the update
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, w = tid >> 5;
  // per-panel face coordinates and kinds, once
  int* pc = reinterpret_cast<int*>(Bp);              // [4][n] (Bp is free until the first panel)
  for (int i = tid; i < n; i += nt) {
    const int pk = idx[q0 + i];
    int c[3];
    face_coords(tt.n, orient[pk], face[pk], c);
    pc[i] = c[0];
    pc[n + i] = c[1];
    pc[2 * n + i] = c[2];
    pc[3 * n + i] = orient[pk] | (kind[pk] << 2);
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += nt) {
    const int i = t / n, j = t - (t / n) * n;
    const int ck[3] = {pc[i], pc[n + i], pc[2 * n + i]};
    const int cl[3] = {pc[j], pc[n + j], pc[2 * n + j]};
    const int oi = pc[3 * n + i] & 3, oj = pc[3 * n + j] & 3;
    const bool E = (pc[3 * n + i] >> 2) == 1;
    double v = a_entry(tt, E, oi, ck, oj, cl);
    if (E && i == j) v += idiag[idx[q0 + i]];
    S[i * ld + j] = (float)v;
  }
  for (int i = tid; i < n; i += nt) used[i] = 0;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n && !fail; k0 += kGJPanel) {
    const int nbp = min(kGJPanel, n - k0);
    for (int kk = 0; kk < nbp; ++kk) {
      const int k = k0 + kk, par = k & 1;
      if (w == kk) {                                 // pivot search by the owner of column k
        float best = -1.0f;
        int bi = n;
        for (int i = lane; i < n; i += 32) {
          const float v = S[i * ld + k];
          colb[par][i] = v;
          if (!used[i] && fabsf(v) > best) { best = fabsf(v); bi = i; }
        }
        for (int d = 16; d > 0; d >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, d);
          const int oi = __shfl_down_sync(0xffffffffu, bi, d);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        __syncwarp();
        if (lane == 0) {
          if (!(best > 0.0f) || bi >= n) {
            fail = 1;
            bi = 0;
          }
          prow[par] = bi;
          pinv[par] = 1.0f / colb[par][bi];
          perm[k] = bi;
          used[bi] = 1;
          pan_rows[kk] = bi;
        }
      }
      __syncthreads();
      if (fail) break;                               // uniform: read after the barrier
      const int p = prow[par];
      const float ip = pinv[par];
      if (w < nbp) {                                 // warp w updates panel column k0 + w
        const int c = k0 + w;
        const float sp = S[p * ld + c];
        __syncwarp();                                // every lane has row p's old value
        const float rpc = (c == k ? 1.0f : sp) * ip;
        for (int i = lane; i < n; i += 32) {
          float* e = S + i * ld + c;
          if (i == p) *e = rpc;
          else *e = (c == k ? 0.0f : *e) - colb[par][i] * rpc;
        }
      }
    }
    __syncthreads();
    if (fail) break;
    // rank-nbp update of the columns outside the panel
    for (int t = tid; t < nbp * n; t += nt) {
      const int r = t / n, j = t - (t / n) * n;
      Bp[r * ld + j] = S[pan_rows[r] * ld + j];
    }
    __syncthreads();
    const int nwarps = nt >> 5;
    for (int i0 = 4 * w; i0 < n; i0 += 4 * nwarps) {
      float acc[4][8];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[q][e] = 0.0f;
      auto rank1 = [&](int r) {
        float av[4], bv[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) av[q] = (i0 + q < n) ? S[(i0 + q) * ld + k0 + r] : 0.0f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = lane + 32 * e;
          bv[e] = j < n ? Bp[r * ld + j] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[q][e] += av[q] * bv[e];
      };
      if (nbp == kGJPanel) {
#pragma unroll
        for (int r = 0; r < kGJPanel; ++r) rank1(r);
      } else {
        for (int r = 0; r < nbp; ++r) rank1(r);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q;
        if (i >= n) continue;
        bool in_pan = false;
        for (int r = 0; r < nbp; ++r) in_pan = in_pan || pan_rows[r] == i;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = lane + 32 * e;
          if (j < n && (j < k0 || j >= k0 + nbp)) {
            float* x = S + i * ld + j;
            *x = (in_pan ? 0.0f : *x) + acc[q][e];
          }
        }
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) atomicExch(status, 1);
    return;
  }
  for (int k = tid; k < n; k += nt) qinv[perm[k]] = k;
  __syncthreads();
  const int64_t o = uoff[u];
  for (int t = tid; t < n * n; t += nt) {
    const int i = t / n, j = t - (t / n) * n;
    const float v = S[i * ld + j];
    const int64_t d = o + (int64_t)qinv[i] * n + perm[j];
    inv_f[d] = v;
    inv_d[d] = (double)v;
  }
}

// Gauss-Jordan with partial pivoting on [A | I] -> [I | A^-1], one launch
// per elimination step c.  The 2n columns of every block are split into
// slabs of kGJCols columns, one CTA each, so a step touches each block with
// many SMs.  The pivot column c (needed by every slab) is read from `pin`,
// the copy the owner of column c wrote in the previous step; the owner of
// column c+1 writes its updated column to `pout` for the next step.  Step c
// with pivot row pr (old values; mult = column c, piv = mult[pr]):
//   new row c   = old row pr / piv
//   new row pr  = old row c - mult[c] * (new row c)       (pr != c)
//   other row r = old row r - mult[r] * (new row c)
constexpr int kGJCols = 16;

__global__ void k_gj_step(int c, const int32_t* __restrict__ urep, const int32_t* __restrict__ offs,
                          const int64_t* __restrict__ aoff, const int64_t* __restrict__ poff,
                          double* __restrict__ aug, const double* __restrict__ pin,
                          double* __restrict__ pout, int* __restrict__ status) {
  extern __shared__ double gsm[];
  const int u = blockIdx.y;
  const int gb = urep[u];
  const int n = offs[gb + 1] - offs[gb];
  if (c >= n) return;
  const int w = 2 * n;
  const int j0 = blockIdx.x * kGJCols;
  if (j0 >= w) return;
  const int j1 = min(w, j0 + kGJCols);
  double* Mx = aug + aoff[u];
  double* mult = gsm;                 // [n]
  double* prow = gsm + n;             // [kGJCols]
  double* crow = prow + kGJCols;      // [kGJCols]
  __shared__ double red_v[256];
  __shared__ int red_i[256];
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    mult[r] = (c == 0) ? Mx[(int64_t)r * w] : pin[poff[u] + r];
  __syncthreads();
  double best = -1.0;
  int bi = n;
  for (int r = c + threadIdx.x; r < n; r += blockDim.x) {
    const double v = fabs(mult[r]);
    if (v > best) { best = v; bi = r; }
  }
  red_v[threadIdx.x] = best;
  red_i[threadIdx.x] = bi;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      const double a = red_v[threadIdx.x], b = red_v[threadIdx.x + st];
      const int ia = red_i[threadIdx.x], ib = red_i[threadIdx.x + st];
      if (b > a || (b == a && ib < ia)) { red_v[threadIdx.x] = b; red_i[threadIdx.x] = ib; }
    }
    __syncthreads();
  }
  const int pr = red_i[0];
  const double piv = mult[pr < n ? pr : c];
  if (!(red_v[0] > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(status, 1);
    return;
  }
  const double ipiv = 1.0 / piv;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    prow[j - j0] = Mx[(int64_t)pr * w + j] * ipiv;
    crow[j - j0] = Mx[(int64_t)c * w + j];
  }
  __syncthreads();
  const int cw = j1 - j0;
  const double mc = mult[c];
  for (int t = threadIdx.x; t < n * cw; t += blockDim.x) {
    const int r = t / cw, jj = t % cw;
    const int64_t at = (int64_t)r * w + j0 + jj;
    const double pj = prow[jj];
    if (r == c) Mx[at] = pj;
    else if (r == pr) Mx[at] = crow[jj] - mc * pj;
    else Mx[at] -= mult[r] * pj;
  }
  __syncthreads();
  const int nc = c + 1;
  if (nc < n && nc >= j0 && nc < j1)
    for (int r = threadIdx.x; r < n; r += blockDim.x) pout[poff[u] + r] = Mx[(int64_t)r * w + nc];
}

__global__ void k_extract_inv(const int32_t* urep, const int32_t* offs, const int64_t* aoff,
                              const int64_t* uoff, const double* aug, double* inv_d, float* inv_f) {
  const int u = blockIdx.x;
  const int gb = urep[u];
  const int n = offs[gb + 1] - offs[gb];
  const double* Mx = aug + aoff[u];
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    double v = Mx[(int64_t)i * 2 * n + n + j];
    inv_d[uoff[u] + t] = v;
    inv_f[uoff[u] + t] = (float)v;
  }
}

__global__ void k_diag_scale(int64_t N, int mode, const int8_t* kind, const double* idiag,
                             const double* pself_p, const int32_t* inblk, double* dd, float* df) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const double pself = *pself_p;
  double v;
  if (mode == VOXCAP_PRECOND_NONE) v = 1.0;
  else if (mode == VOXCAP_PRECOND_DIAG) v = kind[p] == 0 ? 1.0 / pself : 1.0 / idiag[p];
  else if (inblk && inblk[p]) v = 0.0;
  else v = kind[p] == 1 ? 1.0 / idiag[p] : 1.0 / pself;
  dd[p] = v;
  df[p] = (float)v;
}

__global__ void k_mark_inblk(int64_t total, const int32_t* idx, int32_t* inblk) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < total) inblk[idx[q]] = 1;
}

int build_precond(Handle& h) {
  Precond& P = h.pre;
  P.kind = h.opts.precond;
  for (int a = 0; a < 3; ++a) P.nv[a] = h.opts.nv[a] > 0 ? h.opts.nv[a] : 10;
  const Geom& g = h.g;
  const int64_t N = h.pan.N;
  const int S = h.pan.S;
  VC_TRY(P.dscale_d.alloc((size_t)std::max<int64_t>(N, 1)));
  VC_TRY(P.dscale_f.alloc((size_t)std::max<int64_t>(N, 1)));
  const double* pself = h.toep[0].p;      // self term P'_kk (identical for every orientation)
  const int TB = 256;
  P.nblocks = 0;
  P.nunique = 0;
  P.max_n = 0;
  if (P.kind == VOXCAP_PRECOND_NONE || P.kind == VOXCAP_PRECOND_DIAG || N == 0) {
    k_diag_scale<<<(unsigned)((N + TB - 1) / TB), TB, 0, h.stream>>>(
        N, P.kind, h.pan.kind.p, h.pan.idiag.p, pself, nullptr, P.dscale_d.p, P.dscale_f.p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
    return VOXCAP_OK;
  }
  BoxGeom bg;
  bg.n[0] = g.nx; bg.n[1] = g.ny; bg.n[2] = g.nz;
  for (int a = 0; a < 3; ++a) {
    bg.nv[a] = P.nv[a];
    bg.nb[a] = (bg.n[a] + P.nv[a] - 1) / P.nv[a];
  }
  bg.nbox = (int64_t)bg.nb[0] * bg.nb[1] * bg.nb[2];
  bg.Lx = g.Lx; bg.Ly = g.Ly; bg.Lz = g.Lz;
  P.nbx = bg.nb[0]; P.nby = bg.nb[1]; P.nbz = bg.nb[2];
  const int64_t nboxes = bg.nbox * S;
  P.nboxes = nboxes;
  P.nblocks = nboxes;
  // box -> panels (every panel lies in exactly one box, so N bounds the total)
  VC_TRY(P.blk_off.alloc((size_t)nboxes + 1));
  DBuf<int32_t> tmp;
  VC_TRY(tmp.alloc((size_t)scan_tmp_elems(nboxes + 1) + 8));
  VC_CUDA(cudaMemsetAsync(P.blk_off.p, 0, sizeof(int32_t) * (nboxes + 1), h.stream));
  k_box_count<<<(unsigned)nboxes, TB, 0, h.stream>>>(bg, h.pan.fmap.p, h.pan.kind.p, P.kind, P.blk_off.p); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  VC_TRY(exclusive_scan_i32(P.blk_off.p, nboxes + 1, tmp.p, nullptr, h.stream));
  VC_TRY(P.blk_idx.alloc((size_t)std::max<int64_t>(N, 1)));
  k_box_fill<<<(unsigned)nboxes, TB, 0, h.stream>>>(bg, h.pan.fmap.p, h.pan.kind.p, P.kind, P.blk_off.p,
                                                   P.blk_idx.p); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  // dedup: representatives, their flags (kept) and unique ids (scan of a copy)
  DBuf<uint64_t> hash;
  DBuf<int32_t> rep, meta;                 // meta = [blk_off (nboxes + 1) | is_rep (nboxes)]
  DBuf<int32_t> rep_scan;
  VC_TRY(hash.alloc((size_t)nboxes));
  VC_TRY(rep.alloc((size_t)nboxes));
  VC_TRY(meta.alloc((size_t)2 * nboxes + 1));
  VC_TRY(rep_scan.alloc((size_t)nboxes + 1));
  int32_t* isrep = meta.p + nboxes + 1;
  unsigned nbk = (unsigned)((nboxes + TB - 1) / TB);
  k_box_hash<<<(unsigned)((nboxes * 32 + TB - 1) / TB), TB, 0, h.stream>>>(bg, nboxes, P.blk_off.p, P.blk_idx.p, h.pan.orient.p,
                                       h.pan.face.p, h.pan.kind.p, h.pan.idiag.p, P.kind, hash.p); ::vc::note_launch();
  k_box_rep<<<nbk, TB, 0, h.stream>>>(bg, nboxes, P.blk_off.p, P.blk_idx.p, h.pan.orient.p,
                                      h.pan.face.p, h.pan.kind.p, h.pan.idiag.p, P.kind, hash.p,
                                      rep.p, isrep); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  VC_CUDA(cudaMemcpyAsync(rep_scan.p, isrep, sizeof(int32_t) * nboxes, cudaMemcpyDeviceToDevice, h.stream));
  VC_CUDA(cudaMemsetAsync(rep_scan.p + nboxes, 0, sizeof(int32_t), h.stream));
  VC_TRY(exclusive_scan_i32(rep_scan.p, nboxes + 1, tmp.p, nullptr, h.stream));
  VC_TRY(P.blk_uid.alloc((size_t)nboxes));
  k_box_uid<<<nbk, TB, 0, h.stream>>>(nboxes, rep.p, rep_scan.p, P.blk_off.p, P.blk_uid.p); ::vc::note_launch();
  VC_CUDA(cudaMemcpyAsync(meta.p, P.blk_off.p, sizeof(int32_t) * (nboxes + 1), cudaMemcpyDeviceToDevice,
                          h.stream));
  VC_CUDA(cudaGetLastError());
  // one read-back sizes the inverse storage (a pageable copy waits for the work above)
  std::vector<int32_t> meta_h((size_t)2 * nboxes + 1);
  VC_CUDA(cudaMemcpyAsync(meta_h.data(), meta.p, sizeof(int32_t) * meta_h.size(), cudaMemcpyDeviceToHost,
                          h.stream));
  VC_CUDA(cudaStreamSynchronize(h.stream));
  const int32_t* off_h = meta_h.data();
  const int32_t* isrep_h = meta_h.data() + nboxes + 1;
  const int64_t total = off_h[nboxes];
  std::vector<int32_t> urep_h, urepL_h;
  std::vector<int64_t> uoff_h(1, 0), uoffL_h, aoffL_h(1, 0);
  int max_small = 0, max_large = 0;
  for (int64_t b = 0; b < nboxes; ++b) {
    const int n = off_h[b + 1] - off_h[b];
    P.max_n = std::max(P.max_n, n);
    if (!isrep_h[b]) continue;
    if (n <= kGJTileMax) {
      max_small = std::max(max_small, n);
    } else {
      max_large = std::max(max_large, n);
      urepL_h.push_back((int32_t)b);
      uoffL_h.push_back(uoff_h.back());
      aoffL_h.push_back(aoffL_h.back() + 2 * (int64_t)n * n);
    }
    urep_h.push_back((int32_t)b);
    uoff_h.push_back(uoff_h.back() + (int64_t)n * n);
  }
  const int64_t nuniq = (int64_t)urep_h.size();
  const int64_t nlarge = (int64_t)urepL_h.size();
  P.nunique = nuniq;
  const int64_t inv_elems = uoff_h.back();
  DBuf<int32_t> urep;
  VC_TRY(urep.alloc(std::max<size_t>(urep_h.size(), 1)));
  VC_TRY(P.uoff.alloc(uoff_h.size()));
  VC_TRY(P.inv_d.alloc((size_t)std::max<int64_t>(inv_elems, 1)));
  VC_TRY(P.inv_f.alloc((size_t)std::max<int64_t>(inv_elems, 1)));
  if (nuniq > 0)
    VC_CUDA(cudaMemcpyAsync(urep.p, urep_h.data(), sizeof(int32_t) * urep_h.size(), cudaMemcpyHostToDevice, h.stream));
  VC_CUDA(cudaMemcpyAsync(P.uoff.p, uoff_h.data(), sizeof(int64_t) * uoff_h.size(), cudaMemcpyHostToDevice, h.stream));
  DBuf<int> status;
  VC_TRY(status.alloc(1));
  VC_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), h.stream));
  ToepTabs tt;
  for (int kk = 0; kk < kNumKernels; ++kk) {
    tt.T[kk] = h.toep[kk].p;
    for (int a = 0; a < 3; ++a) tt.d[kk][a] = h.tdims[kk][a];
  }
  tt.n[0] = g.nx; tt.n[1] = g.ny; tt.n[2] = g.nz;
  if (max_small > 0) {
    // blocks of up to kGJTileMax panels: one CTA each, the block in shared memory
    const size_t sm = sizeof(float) * (size_t)(max_small + kGJPanel) * (max_small | 1);
    VC_CUDA(cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_block_inverse<<<(unsigned)nuniq, 1024, sm, h.stream>>>(
        tt, urep.p, P.blk_off.p, P.blk_idx.p, P.uoff.p, h.pan.orient.p, h.pan.face.p, h.pan.kind.p,
        h.pan.idiag.p, P.inv_d.p, P.inv_f.p, status.p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  if (nlarge > 0) {
    // larger blocks: FP64 Gauss-Jordan on [A | I], one launch per elimination step
    DBuf<int32_t> urepL;
    DBuf<int64_t> uoffL, aoffL, poff;
    DBuf<double> aug, pbuf;
    std::vector<int64_t> poff_h(nlarge + 1, 0);
    for (int64_t q = 0; q < nlarge; ++q) poff_h[q + 1] = poff_h[q] + (off_h[urepL_h[q] + 1] - off_h[urepL_h[q]]);
    VC_TRY(urepL.alloc(urepL_h.size()));
    VC_TRY(uoffL.alloc(uoffL_h.size()));
    VC_TRY(aoffL.alloc(aoffL_h.size()));
    VC_TRY(poff.alloc(poff_h.size()));
    VC_TRY(aug.alloc((size_t)aoffL_h.back()));
    VC_TRY(pbuf.alloc((size_t)std::max<int64_t>(2 * poff_h.back(), 1)));
    VC_CUDA(cudaMemcpyAsync(urepL.p, urepL_h.data(), sizeof(int32_t) * urepL_h.size(), cudaMemcpyHostToDevice, h.stream));
    VC_CUDA(cudaMemcpyAsync(uoffL.p, uoffL_h.data(), sizeof(int64_t) * uoffL_h.size(), cudaMemcpyHostToDevice, h.stream));
    VC_CUDA(cudaMemcpyAsync(aoffL.p, aoffL_h.data(), sizeof(int64_t) * aoffL_h.size(), cudaMemcpyHostToDevice, h.stream));
    VC_CUDA(cudaMemcpyAsync(poff.p, poff_h.data(), sizeof(int64_t) * poff_h.size(), cudaMemcpyHostToDevice, h.stream));
    k_assemble<<<(unsigned)nlarge, TB, 0, h.stream>>>(tt, urepL.p, P.blk_off.p, P.blk_idx.p, aoffL.p,
                                                      h.pan.orient.p, h.pan.face.p, h.pan.kind.p,
                                                      h.pan.idiag.p, aug.p); ::vc::note_launch();
    const int slabs = (2 * max_large + kGJCols - 1) / kGJCols;
    const size_t sm = sizeof(double) * ((size_t)max_large + 2 * kGJCols);
    if (sm > 48 * 1024)
      VC_CUDA(cudaFuncSetAttribute(k_gj_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)slabs, (unsigned)nlarge);
    for (int c = 0; c < max_large; ++c) {
      const double* pin = pbuf.p + (c & 1) * poff_h.back();
      double* pout = pbuf.p + ((c + 1) & 1) * poff_h.back();
      k_gj_step<<<grid, TB, sm, h.stream>>>(c, urepL.p, P.blk_off.p, aoffL.p, poff.p, aug.p, pin,
                                            pout, status.p); ::vc::note_launch();
    }
    VC_CUDA(cudaGetLastError());
    k_extract_inv<<<(unsigned)nlarge, TB, 0, h.stream>>>(urepL.p, P.blk_off.p, aoffL.p, uoffL.p, aug.p,
                                                         P.inv_d.p, P.inv_f.p); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  DBuf<int32_t> inblk;
  VC_TRY(inblk.alloc((size_t)std::max<int64_t>(N, 1)));
  VC_CUDA(cudaMemsetAsync(inblk.p, 0, sizeof(int32_t) * std::max<int64_t>(N, 1), h.stream));
  if (total > 0)
    k_mark_inblk<<<(unsigned)((total + TB - 1) / TB), TB, 0, h.stream>>>(total, P.blk_idx.p, inblk.p); ::vc::note_launch();
  k_diag_scale<<<(unsigned)((N + TB - 1) / TB), TB, 0, h.stream>>>(
      N, P.kind, h.pan.kind.p, h.pan.idiag.p, pself, inblk.p, P.dscale_d.p, P.dscale_f.p); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  int st = 0;
  VC_CUDA(cudaMemcpyAsync(&st, status.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
  VC_CUDA(cudaStreamSynchronize(h.stream));
  VC_CHECK(st == 0, VOXCAP_ERR_ARG, "singular preconditioner block");
  return VOXCAP_OK;
}

// ---------------------------------------------------------------- apply
template <typename T>
__global__ void k_pre_diag(int64_t N, int nrhs, const T* __restrict__ ds, const T* __restrict__ r,
                           T* __restrict__ z) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  z[t] = ds[t % N] * r[t];
}

// z_B = R_B r_B for one box (blockIdx.x), one column (blockIdx.y) and the
// rows [32 blockIdx.z, 32 blockIdx.z + 32) of its block; accumulation in T
// (the FP32 inner solve's preconditioner needs no FP64 sums).
constexpr int kPreRows = 32;

template <typename T>
__global__ void k_pre_blocks(int64_t N, const int32_t* __restrict__ offs, const int32_t* __restrict__ idx,
                             const int32_t* __restrict__ uid, const int64_t* __restrict__ uoff,
                             const T* __restrict__ inv, const T* __restrict__ r, T* __restrict__ z) {
  extern __shared__ unsigned char smem_raw[];
  T* rv = reinterpret_cast<T*>(smem_raw);
  const int64_t gb = blockIdx.x;
  const int rhs = blockIdx.y;
  const int q0 = offs[gb];
  const int n = offs[gb + 1] - q0;
  const int i0 = blockIdx.z * kPreRows;
  if (i0 >= n) return;
  const T* Minv = inv + uoff[uid[gb]];
  const T* rr = r + (int64_t)rhs * N;
  T* zz = z + (int64_t)rhs * N;
  for (int j = threadIdx.x; j < n; j += blockDim.x) rv[j] = rr[idx[q0 + j]];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i1 = min(n, i0 + kPreRows);
  for (int i = i0 + wid; i < i1; i += nw) {
    T acc = (T)0;
    const T* row = Minv + (int64_t)i * n;
    for (int j = lane; j < n; j += 32) acc += row[j] * rv[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) zz[idx[q0 + i]] = acc;
  }
}

template <typename T> static const T* dscale_of(const Handle& h);
template <> const float* dscale_of<float>(const Handle& h) { return h.pre.dscale_f.p; }
template <> const double* dscale_of<double>(const Handle& h) { return h.pre.dscale_d.p; }
template <typename T> static const T* inv_of(const Handle& h);
template <> const float* inv_of<float>(const Handle& h) { return h.pre.inv_f.p; }
template <> const double* inv_of<double>(const Handle& h) { return h.pre.inv_d.p; }

template <typename T>
int precond_apply(Handle& h, const T* r, T* z, int nrhs) {
  const int64_t N = h.pan.N;
  const int TB = 256;
  if (N == 0) return VOXCAP_OK;
  k_pre_diag<T><<<(unsigned)((N * nrhs + TB - 1) / TB), TB, 0, h.stream>>>(N, nrhs, dscale_of<T>(h), r, z); ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  const Precond& P = h.pre;
  if ((P.kind == VOXCAP_PRECOND_BDD || P.kind == VOXCAP_PRECOND_BD) && P.nblocks > 0 && P.max_n > 0) {
    size_t sm = sizeof(T) * (size_t)P.max_n;
    if (sm > 48 * 1024)
      VC_CUDA(cudaFuncSetAttribute(k_pre_blocks<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)P.nblocks, nrhs, (unsigned)((P.max_n + kPreRows - 1) / kPreRows));
    k_pre_blocks<T><<<grid, 128, sm, h.stream>>>(N, P.blk_off.p, P.blk_idx.p, P.blk_uid.p, P.uoff.p,
                                                inv_of<T>(h), r, z); ::vc::note_launch();
    VC_CUDA(cudaGetLastError());
  }
  return VOXCAP_OK;
}

template int precond_apply<float>(Handle&, const float*, float*, int);
template int precond_apply<double>(Handle&, const double*, double*, int);

}  // namespace vc
