// z pass of the forward FP32 product (Eqs. 9-12) on compiled two-stage
// plans Mz = RA * RB: forward z transforms of the three charge spectra, the
// spectral multiply-accumulate with the 15 real kernel spectra (6 potential,
// 9 normal-field blocks; Eq. 12 folds the other three potential blocks) and
// the inverse z transforms back to the N_z+1 planes the panels need.
//
// A CTA (RA * TX threads) takes TX consecutive (ky, kx) columns of one batch
// item.  Stage A (radix RA) reads the N_z+1 non-zero planes of the three
// input grids from HBM and fills the shared buffer [Mz][3][TX]; each thread
// then holds the RB frequencies kz = j + RA r of its column for all three
// grids (last forward stage, parked in a second shared buffer), multiplies
// them with the kernel spectra -- read as one 64-byte record of the 15 real
// kernels per frequency, side by side -- and runs the first inverse stage;
// the outputs go through the first buffer in two halves (potential grids,
// then field grids) to the last inverse stage (radix RA), which writes
// planes z <= N_z to HBM.
#include "fast.cuh"

namespace vc {

namespace {

using fast::C;

// test / source orientation of kernel kk and its fold signs R(M-k) = +-R(k)
// along y (a = 1) and z (a = 2), as compile-time constants
constexpr int ktest(int kk) {
  return (kk == 0 || kk == 3 || kk == 4 || kk == 6 || kk == 9 || kk == 10) ? 0
         : (kk == 1 || kk == 5 || kk == 7 || kk == 11 || kk == 12)         ? 1
                                                                           : 2;
}
constexpr int ksrc(int kk) {
  return (kk == 0 || kk == 6 || kk == 12 || kk == 13) ? 0 : (kk == 1 || kk == 3 || kk == 7 || kk == 9 || kk == 14) ? 1 : 2;
}
constexpr bool kflip(int kk, int a) {
  return ktest(kk) == ksrc(kk) ? (kk >= 6 && a == ktest(kk))
                               : (a == ktest(kk) ? kk < 6 : a == ksrc(kk));
}

// kernel value kk of a frequency record in HBM (16 floats, kernels side by
// side) with the fold signs of the frequency applied
template <int KK>
__device__ __forceinline__ float kval(const float* rec, float sy, float sz) {
  float v = __ldg(rec + KK);
  if constexpr (kflip(KK, 1)) v *= sy;
  if constexpr (kflip(KK, 2)) v *= sz;
  return v;
}

template <int RA, int RB, int TX>
__global__ void __launch_bounds__(RA * TX, 2) k_zpass_fast(Geom g, C* __restrict__ data,
                                                          const float4* __restrict__ specv,
                                                          const C* __restrict__ twf, int twn_f, int offB,
                                                          const C* __restrict__ twv, int twn_v, int offA,
                                                          const C* __restrict__ phz, int nbatch) {
  constexpr int L = RA * RB;
  constexpr int NT = RA * TX;
  constexpr int LD = 3 * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);      // [L][3][TX]: z lines between the stages
  C* S = buf + L * LD;                          // [3][RB][NT]: each thread's charge spectra
  C* tf = S + 3 * RB * NT;
  C* tv = tf + twn_f;
  C* ph = tv + twn_v;
  fast::load_table<NT>(tf, twf, twn_f);
  fast::load_table<NT>(tv, twv, twn_v);
  fast::load_table<NT>(ph, phz, L);
  const int H = g.Hx;
  const int b = blockIdx.x % nbatch;                      // batch items of a tile run together
  const int64_t zstride = (int64_t)g.My * H;              // one z plane [My][H]
  const int64_t q0 = (int64_t)(blockIdx.x / nbatch) * TX; // first column q = ky * H + kx
  const int64_t gstride = (int64_t)g.Lz * zstride;
  C* base = data + (int64_t)b * 6 * gstride + q0;
  const int ncol = (int)min((int64_t)TX, zstride - q0);
  const int Lz = g.Lz;
  __syncthreads();

  // ---- stage A: forward radix RA of the three input grids, HBM -> buffer
  fast::stage<L, RA, 1, LD, NT, false>(
      tf,
      [&](int line, int z) -> C {
        const int grid = line / TX, c = line % TX;
        C v = mk<C>(0.f, 0.f);
        if (c < ncol && z < Lz) v = base[grid * gstride + z * zstride + c];
        return v;
      },
      [&](int line, int pos, C v) { buf[pos * LD + line] = v; });
  __syncthreads();

  // ---- last forward stage (radix RB): thread (j, c) gets kz = j + RA r
  const int t = threadIdx.x;
  const int j = t / TX, c = t % TX;
  const bool col_ok = c < ncol;
#pragma unroll
  for (int be = 0; be < 3; ++be) {
    C v[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) v[r] = buf[(j + r * RA) * LD + be * TX + c];
    fast::twiddle<RB, false>(v, tf + offB, j);
    dft<RB, C>(v, false);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (be == 2) v[r] = cmul(v[r], ph[j + r * RA]);   // half-voxel shift of z grids
      S[(be * RB + r) * NT + t] = v[r];
    }
  }
  __syncthreads();                                      // the buffer takes the outputs now

  // frequency records of the column: (kz folded, ky folded, kx)
  const int64_t q = q0 + c;
  const int ky = col_ok ? (int)(q / H) : 0;
  const int kx = col_ok ? (int)(q - (int64_t)ky * H) : 0;
  const bool fy = ky > g.My / 2;
  const float sy = fy ? -1.f : 1.f;
  const int64_t rec0 = (int64_t)(fy ? g.My - ky : ky) * H + kx;
  const int64_t zrec = (int64_t)g.Oy * H;

#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    // potential outputs (half 0: kernels 0..5, Eq. 12 pairs shared) or
    // normal-field outputs (half 1: kernels 6..14, times -i), one output
    // grid at a time
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      C o[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int kz = j + r * RA;
        const bool fz = kz > L / 2;
        const float sz = fz ? -1.f : 1.f;
        const float* rec = reinterpret_cast<const float*>(specv) + ((int64_t)(fz ? L - kz : kz) * zrec + rec0) * 16;
        float k0 = 0.f, k1 = 0.f, k2 = 0.f;
        if (col_ok) {
          if (half == 0) {       // P^{ab}: xx yy zz xy xz yz
            if (al == 0) { k0 = kval<0>(rec, sy, sz); k1 = kval<3>(rec, sy, sz); k2 = kval<4>(rec, sy, sz); }
            if (al == 1) { k0 = kval<3>(rec, sy, sz); k1 = kval<1>(rec, sy, sz); k2 = kval<5>(rec, sy, sz); }
            if (al == 2) { k0 = kval<4>(rec, sy, sz); k1 = kval<5>(rec, sy, sz); k2 = kval<2>(rec, sy, sz); }
          } else {               // E^{ab}: xx yy zz xy xz yz yx zx zy
            if (al == 0) { k0 = kval<6>(rec, sy, sz); k1 = kval<9>(rec, sy, sz); k2 = kval<10>(rec, sy, sz); }
            if (al == 1) { k0 = kval<12>(rec, sy, sz); k1 = kval<7>(rec, sy, sz); k2 = kval<11>(rec, sy, sz); }
            if (al == 2) { k0 = kval<13>(rec, sy, sz); k1 = kval<14>(rec, sy, sz); k2 = kval<8>(rec, sy, sz); }
          }
        }
        const C Q0 = S[(0 * RB + r) * NT + t], Q1 = S[(1 * RB + r) * NT + t], Q2 = S[(2 * RB + r) * NT + t];
        C acc;
        acc.x = fmaf(Q0.x, k0, fmaf(Q1.x, k1, Q2.x * k2));
        acc.y = fmaf(Q0.y, k0, fmaf(Q1.y, k1, Q2.y * k2));
        o[r] = half == 0 ? acc : cmul_mi(acc);
      }
      if (al == 2) {
#pragma unroll
        for (int r = 0; r < RB; ++r) o[r] = cmul(o[r], cconj(ph[j + r * RA]));
      }
      dft<RB, C>(o, true);                               // first inverse stage (radix RB, no twiddles)
#pragma unroll
      for (int r = 0; r < RB; ++r) buf[(j * RB + r) * LD + al * TX + c] = o[r];
    }
    __syncthreads();
    // ---- last inverse stage (radix RA), buffer -> HBM, planes z < Lz
    fast::stage<L, RA, RB, LD, NT, true>(
        tv + offA, [&](int line, int pos) -> C { return buf[pos * LD + line]; },
        [&](int line, int z, C v) {
          const int grid = line / TX + 3 * half, cc = line % TX;
          if (cc < ncol && z < Lz) base[grid * gstride + z * zstride + cc] = v;
        });
    __syncthreads();
  }
}

template <int RA, int RB, int TX>
int launch_z(const Handle& h, C* data, int B, cudaStream_t st) {
  const Geom& g = h.g;
  const Plan1D<float2>& pz = h.pzf[0];
  const Plan1D<float2>& pv = h.pzfr[0];
  constexpr int L = RA * RB;
  VC_CHECK(h.spec_v.p != nullptr, VOXCAP_ERR_UNSUPPORTED, "interleaved spectra missing for the z pass");
  const size_t sm = ((size_t)L * 3 * TX + (size_t)3 * RB * RA * TX + pz.twn + pv.twn + L) * sizeof(C);
  const int64_t cols = (int64_t)g.My * g.Hx;
  const int64_t tiles = (cols + TX - 1) / TX;
  VC_CHECK(tiles * B < ((int64_t)1 << 31), VOXCAP_ERR_UNSUPPORTED, "grid too large for the z pass");
  auto kern = k_zpass_fast<RA, RB, TX>;
  VC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)(tiles * B), RA * TX, sm, st>>>(g, data, reinterpret_cast<const float4*>(h.spec_v.p), pz.stw,
                                                   pz.twn, pz.twoff[1], pv.stw, pv.twn, pv.twoff[1], h.phf[2], B);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

}  // namespace

bool fast_z_ok(const Handle& h) {
  const Plan1D<float2>& p = h.pzf[0];
  return p.nst == 2 && p.radix[1] == 9 && (p.radix[0] == 16 || p.radix[0] == 8 || p.radix[0] == 4);
}

int fast_zpass(const Handle& h, float2* data, int B, cudaStream_t st) {
  const Plan1D<float2>& p = h.pzf[0];
  if (p.nst == 2 && p.radix[1] == 9) {
    if (p.radix[0] == 16) return launch_z<16, 9, 16>(h, data, B, st);
    if (p.radix[0] == 8) return launch_z<8, 9, 16>(h, data, B, st);
    if (p.radix[0] == 4) return launch_z<4, 9, 16>(h, data, B, st);
  }
  set_error("no compiled z-pass plan for this length");
  return VOXCAP_ERR_UNSUPPORTED;
}

}  // namespace vc
