// The z pass of the FFT products (Eqs. 9-11): z transforms of the charge
// spectra, the spectral multiply-accumulate with the 15 kernel spectra
// (Eq. 12 folds the other three potential blocks), and the inverse z
// transforms.  Included by one translation unit per precision and direction.
#pragma once
#include <algorithm>

#include "internal.h"

namespace vc {

// fold sign of kernel kk along axis a: R(M-k) = sig * R(k)
inline int fold_sign(int kk, int a) {
  const int te = ker_test(kk), so = ker_src(kk);
  const bool E = kk >= 6;
  if (te == so) return (E && a == te) ? -1 : 1;
  if (a == te) return E ? 1 : -1;
  if (a == so) return -1;
  return 1;
}

// index of the potential block of an unordered orientation pair, and of the
// field block of an ordered (test, source) pair
__device__ __forceinline__ int pidx(int a, int b) {
  if (a == b) return a;
  int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}
__device__ __forceinline__ int eidx(int a, int b) {
  if (a == b) return 6 + a;
  if (a == 0) return b == 1 ? 9 : 10;
  if (a == 1) return b == 2 ? 11 : 12;
  return b == 0 ? 13 : 14;
}


// ------------------------------------------------------------------ zmac
// data: [B][6][Lz][My][H] (in place).  Forward reads grids 0..2, writes 0..5
// (potential x,y,z then field x,y,z).  Adjoint reads 0..5 (conductor-source
// x,y,z then dielectric-source x,y,z) and writes 0..2.
//
// One CTA transforms the z lines of TX = 2^tx_sh consecutive (ky, kx) columns
// (a z plane is [My][H], so column q = ky * H + kx is contiguous).
// The first forward stage reads its inputs straight from global memory
// (planes z >= Lz are the zero padding and are not read), the last forward
// stage (radix RL), the spectral multiply-accumulate and the first stage of
// the inverse transform (plan `pv`, the forward radices in reverse order, so
// it starts with RL on the same RL frequencies) run on one thread's
// registers, and the last inverse stage writes planes z < Lz straight back.
// Shared memory holds one line buffer (element (line, pos) at pos * LD + line,
// LD = grids * TX) plus a second one when middle stages need ping-pong.  The
// fused step works in place: every thread reads its inputs, the block
// synchronises, then the outputs are written; this needs one item per thread
// (blockDim >= (Mz / RL) * TX, guaranteed by the launch).

// spectral factor of kernel kk at (kx, folded ky, folded kz); bit kk of
// `neg` set when the folds along y and z flip its sign
template <typename T>
__device__ __forceinline__ T spec_at(const T* __restrict__ spec, int64_t Otot, int kk, int idx,
                                     uint32_t neg) {
  const T v = __ldg(spec + kk * Otot + idx);
  return ((neg >> kk) & 1u) ? -v : v;
}

template <typename T, bool ADJ, int RL>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_zmac(Geom g, C_t<T>* __restrict__ data, const T* __restrict__ spec,
                                              Plan1D<C_t<T>> pf, Plan1D<C_t<T>> pv,
                                              const C_t<T>* __restrict__ phz, int tx_sh, int nbatch,
                                              uint32_t neg_y, uint32_t neg_z) {
  using C = C_t<T>;
  extern __shared__ unsigned char smem_raw[];
  constexpr int GI = ADJ ? 6 : 3;
  constexpr int GO = ADJ ? 3 : 6;
  const int TX = 1 << tx_sh;
  const int M = g.Mz, H = g.Hx;
  const int nst = pf.nst;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* alt = buf + (size_t)M * 6 * TX;
  C* twf = alt + (nst >= 3 ? (size_t)M * 6 * TX : 0);
  C* twv = twf + pf.twn;
  load_twiddles(twf, pf);
  load_twiddles(twv, pv);
  const int b = blockIdx.x % nbatch;                    // batch items of one tile run together
  const int64_t zstride = (int64_t)g.My * H;            // one z plane: [My][H], contiguous
  const int q0 = (blockIdx.x / nbatch) * TX;            // first (ky, kx) column: q = ky * H + kx
  const int64_t gstride = (int64_t)g.Lz * zstride;      // one grid of one batch item
  C* base = data + (int64_t)b * 6 * gstride + q0;
  const int ncol = (int)min((int64_t)TX, zstride - q0); // valid columns of this tile
  const int LDI = GI * TX, LDO = GO * TX;
  const FastDiv fLDI = make_fastdiv((uint32_t)LDI), fLDO = make_fastdiv((uint32_t)LDO);
  const int Lz = g.Lz;
  auto gload = [&](int line, int z) -> C {
    const int grid = line >> tx_sh, c = line & (TX - 1);
    C v = mk<C>((T)0, (T)0);
    if (c < ncol && z < Lz) v = base[grid * gstride + z * zstride + c];
    return v;
  };
  auto gstore = [&](int line, int z, C v) {
    const int grid = line >> tx_sh, c = line & (TX - 1);
    if (c < ncol && z < Lz) base[grid * gstride + z * zstride + c] = v;
  };
  __syncthreads();

  // ---- forward stages up to the last one
  C* src = buf;
  C* dst = alt;
  const int nb = M / RL;                                // butterflies of the fused stage
  if (nst >= 2) {
    stage_io(pf, 0, twf, LDI, fLDI, false, gload,
             [&](int line, int pos, C v) { buf[pos * LDI + line] = v; });
    __syncthreads();
    for (int s = 1; s < nst - 1; ++s) {
      stage_io(pf, s, twf, LDI, fLDI, false,
               [&](int line, int pos) { return src[pos * LDI + line]; },
               [&](int line, int pos, C v) { dst[pos * LDI + line] = v; });
      __syncthreads();
      C* t = src; src = dst; dst = t;
    }
  }

  // ---- fused: last forward stage, multiply-accumulate, first inverse stage
  const int t = threadIdx.x;
  const bool act = t < (nb << tx_sh);
  const int j = t >> tx_sh, c = t & (TX - 1);
  const bool col_ok = act && c < ncol;
  const C* twl = twf + pf.twoff[nst - 1];               // last forward stage: Ns = nb, k = j
  auto fin = [&](int grid, int r) -> C {
    const int z = j + r * nb;
    if (nst == 1) return gload(grid * TX + c, z);
    return src[z * LDI + grid * TX + c];
  };
  auto fwd_line = [&](int grid, C* v) {
#pragma unroll
    for (int r = 0; r < RL; ++r) v[r] = fin(grid, r);
    if (nst > 1 && nb > 1) {
#pragma unroll
      for (int r = 1; r < RL; ++r) v[r] = cmul(v[r], twl[j * (RL - 1) + r - 1]);
    }
    dft<RL, C>(v, false);
    if (grid % 3 == 2) {                                // half-voxel shift of z grids
#pragma unroll
      for (int r = 0; r < RL; ++r) v[r] = cmul(v[r], phz[j + r * nb]);
    }
  };
  const int64_t Otot = (int64_t)H * g.Oy * g.Oz;
  const int q = q0 + c;
  const int ky = col_ok ? q / H : 0;
  const int kx = q - ky * H;
  const bool fy = ky > g.My / 2;
  const int kyf = fy ? g.My - ky : ky;
  // spectral index and fold-sign mask of frequency kz = j + r nb (recomputed
  // where used: a few integer operations, no registers held across the MAC)
  const uint32_t negy = fy ? neg_y : 0u;
  const int kcol = kyf * H + kx;
  auto sidx = [&](int r) -> int {
    const int kz = j + r * nb;
    return ((kz > M / 2 ? M - kz : kz) * g.Oy) * H + kcol;
  };
  auto sneg = [&](int r) -> uint32_t { return negy ^ ((j + r * nb) > M / 2 ? neg_z : 0u); };
  auto put = [&](int grid, C* o) {                      // inverse first stage (Ns = 1) and store
    if (grid % 3 == 2) {
#pragma unroll
      for (int r = 0; r < RL; ++r) o[r] = cmul(o[r], cconj(phz[j + r * nb]));
    }
    dft<RL, C>(o, true);
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      if (nst == 1) gstore(grid * TX + c, j * RL + r, o[r]);
      else src[(j * RL + r) * LDO + grid * TX + c] = o[r];
    }
  };
  if (!ADJ) {
    C in[3][RL];
    if (act) {
#pragma unroll
      for (int be = 0; be < 3; ++be) fwd_line(be, in[be]);
    }
    __syncthreads();                                    // all inputs read before the outputs land
    if (act) {
#pragma unroll
      for (int al = 0; al < 3; ++al) {
        C o[RL];
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          C acc = mk<C>((T)0, (T)0);
          if (col_ok) {
#pragma unroll
            for (int be = 0; be < 3; ++be)
              acc = cadd(acc, cscale(in[be][r], spec_at(spec, Otot, pidx(al, be), sidx(r), sneg(r))));
          }
          o[r] = acc;
        }
        put(al, o);
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          C acc = mk<C>((T)0, (T)0);
          if (col_ok) {
#pragma unroll
            for (int be = 0; be < 3; ++be)
              acc = cadd(acc, cscale(in[be][r], spec_at(spec, Otot, eidx(al, be), sidx(r), sneg(r))));
          }
          o[r] = cmul_mi(acc);
        }
        put(3 + al, o);
      }
    }
  } else {
    C o[3][RL];
#pragma unroll
    for (int be = 0; be < 3; ++be)
#pragma unroll
      for (int r = 0; r < RL; ++r) o[be][r] = mk<C>((T)0, (T)0);
    if (act) {
#pragma unroll 1
      for (int gi = 0; gi < 6; ++gi) {
        C v[RL];
        fwd_line(gi, v);
        if (!col_ok) continue;
        const int al = gi % 3;
#pragma unroll
        for (int be = 0; be < 3; ++be)
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            if (gi < 3) {
              o[be][r] = cadd(o[be][r], cscale(v[r], spec_at(spec, Otot, pidx(al, be), sidx(r), sneg(r))));
            } else {
              o[be][r] = cadd(o[be][r], cmul_pi(cscale(v[r], spec_at(spec, Otot, eidx(al, be), sidx(r), sneg(r)))));
            }
          }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int be = 0; be < 3; ++be) put(be, o[be]);
    }
  }
  if (nst == 1) return;
  __syncthreads();

  // ---- inverse stages after the first one
  for (int s = 1; s < nst - 1; ++s) {
    stage_io(pv, s, twv, LDO, fLDO, true,
             [&](int line, int pos) { return src[pos * LDO + line]; },
             [&](int line, int pos, C v) { dst[pos * LDO + line] = v; });
    __syncthreads();
    C* tt = src; src = dst; dst = tt;
  }
  stage_io(pv, nst - 1, twv, LDO, fLDO, true,
           [&](int line, int pos) { return src[pos * LDO + line]; }, gstore);
}

template <typename T> inline const Plan1D<C_t<T>>& zplan(const Handle& h, int v, bool rev);
template <> inline const Plan1D<float2>& zplan<float>(const Handle& h, int v, bool rev) {
  return rev ? h.pzfr[v] : h.pzf[v];
}
template <> inline const Plan1D<double2>& zplan<double>(const Handle& h, int v, bool rev) {
  return rev ? h.pzdr[v] : h.pzd[v];
}

template <typename T, bool ADJ>
int zmac_launch(const Handle& h, C_t<T>* data, int B, cudaStream_t st, int var, int tx_req) {
  using C = C_t<T>;
  const Geom& g = h.g;
  if (var < 0) var = sizeof(T) == 4 ? h.zvar : 0;
  if (var >= h.nzvar) var = 0;
  if (tx_req < 0 && sizeof(T) == 4) tx_req = h.ztx;
  const Plan1D<C>& pz = zplan<T>(h, var, false);
  const Plan1D<C>& pzr = zplan<T>(h, var, true);
  const int RL = pz.radix[pz.nst - 1];
  const int nb = g.Mz / RL;
  const int nbuf = pz.nst >= 3 ? 2 : 1;
  auto fits = [&](int sh) {
    return (nb << sh) <= 256 && (size_t)nbuf * g.Mz * 6 * (1 << sh) * sizeof(C) <= 110 * 1024;
  };
  int tx_sh = 4;
  if (tx_req >= 0 && tx_req <= 4 && fits(tx_req)) {
    tx_sh = tx_req;
  } else {
    while (tx_sh > 0 && !fits(tx_sh)) --tx_sh;
  }
  VC_CHECK((nb << tx_sh) <= 256, VOXCAP_ERR_UNSUPPORTED, "z transform too long for the fused z pass");
  const int TX = 1 << tx_sh;
  const int TB = std::max(64, ((nb << tx_sh) + 31) / 32 * 32);
  const size_t sm = ((size_t)nbuf * g.Mz * 6 * TX + pz.twn + pzr.twn) * sizeof(C);
  uint32_t neg_y = 0, neg_z = 0;
  for (int kk = 0; kk < kNumKernels; ++kk) {
    if (fold_sign(kk, 1) < 0) neg_y |= 1u << kk;
    if (fold_sign(kk, 2) < 0) neg_z |= 1u << kk;
  }
  const int64_t cols = (int64_t)g.My * g.Hx;
  const int64_t tiles = (cols + TX - 1) / TX;
  VC_CHECK(tiles * B < ((int64_t)1 << 31) && (int64_t)g.Hx * g.Oy * g.Oz < ((int64_t)1 << 31),
           VOXCAP_ERR_UNSUPPORTED, "grid too large for the z pass");
  // blockIdx.x = tile * B + item: the items of a tile are adjacent and share its spectra in L2
  dim3 grid((unsigned)(tiles * B));
#define VC_ZMAC(R)                                                                              \
  case R:                                                                                       \
    VC_TRY(set_smem(k_zmac<T, ADJ, R>, sm));                                                    \
    k_zmac<T, ADJ, R><<<grid, TB, sm, st>>>(g, data, spec_of<T>(h), pz, pzr, phase_of<T>(h, 2),  \
                                            tx_sh, B, neg_y, neg_z);                               \
    break;
  switch (RL) {
    VC_ZMAC(2) VC_ZMAC(3) VC_ZMAC(4) VC_ZMAC(5) VC_ZMAC(7) VC_ZMAC(8) VC_ZMAC(9)
    default: VC_CHECK(false, VOXCAP_ERR_UNSUPPORTED, "unsupported last z radix");
  }
#undef VC_ZMAC
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

}  // namespace vc
