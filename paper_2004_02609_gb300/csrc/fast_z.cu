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
// them with the real kernel spectra and runs the first inverse stage;
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

// kernel block of output grid AL and source grid BE: potential (HALF 0:
// P^{ab} xx yy zz xy xz yz, the symmetric pairs shared) or normal field
// (HALF 1: E^{ab} xx yy zz xy xz yz yx zx zy)
constexpr int kidx(int half, int al, int be) {
  return half == 0 ? (al == be ? al : (al + be == 1 ? 3 : (al + be == 2 ? 4 : 5)))
                   : (al == be ? 6 + al
                               : (al == 0 ? (be == 1 ? 9 : 10) : (al == 1 ? (be == 2 ? 11 : 12) : (be == 0 ? 13 : 14))));
}

// One output grid AL of half HALF at the thread's RB frequencies: the 3 RB
// kernel values (read together; consecutive columns of a warp read
// consecutive floats of one kernel's octant), the fold signs,
// the sum over the 3 source grids, the output half-voxel phase of z grids,
// the first inverse stage, and the store to the line buffer.
template <int HALF, int AL, int RA, int RB, int NT, int TX, int LD>
__device__ __forceinline__ void mac_out(const float* __restrict__ spec, int otot, const int* off, bool col_ok,
                                        float sy, const C* S, int t, int j, int c, const C* ph, C* buf) {
  constexpr int L = RA * RB;
  constexpr int K0 = kidx(HALF, AL, 0), K1 = kidx(HALF, AL, 1), K2 = kidx(HALF, AL, 2);
  float kv[RB][3];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    kv[r][0] = col_ok ? __ldg(spec + K0 * otot + off[r]) : 0.f;
    kv[r][1] = col_ok ? __ldg(spec + K1 * otot + off[r]) : 0.f;
    kv[r][2] = col_ok ? __ldg(spec + K2 * otot + off[r]) : 0.f;
  }
  C o[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const float sz = (j + r * RA) > L / 2 ? -1.f : 1.f;
    const float k0 = kv[r][0] * (kflip(K0, 1) ? sy : 1.f) * (kflip(K0, 2) ? sz : 1.f);
    const float k1 = kv[r][1] * (kflip(K1, 1) ? sy : 1.f) * (kflip(K1, 2) ? sz : 1.f);
    const float k2 = kv[r][2] * (kflip(K2, 1) ? sy : 1.f) * (kflip(K2, 2) ? sz : 1.f);
    const C Q0 = S[(0 * RB + r) * NT + t], Q1 = S[(1 * RB + r) * NT + t], Q2 = S[(2 * RB + r) * NT + t];
    C acc;
    acc.x = fmaf(Q0.x, k0, fmaf(Q1.x, k1, Q2.x * k2));
    acc.y = fmaf(Q0.y, k0, fmaf(Q1.y, k1, Q2.y * k2));
    o[r] = HALF == 0 ? acc : cmul_mi(acc);
    if (AL == 2) o[r] = cmul(o[r], cconj(ph[j + r * RA]));
  }
  dft<RB, C>(o, true);                                   // first inverse stage (radix RB, no twiddles)
#pragma unroll
  for (int r = 0; r < RB; ++r) buf[(j * RB + r) * LD + AL * TX + c] = o[r];
}

template <int RA, int RB, int TX>
__global__ void __launch_bounds__(RA * TX, 2) k_zpass_fast(Geom g, C* __restrict__ data,
                                                          const float* __restrict__ spec, int otot,
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

  // spectral index of the column's frequencies (kz folded, ky folded, kx)
  // in a kernel's octant [Oz][Oy][Hx]; 32-bit (the launch checks the size)
  const int64_t q = q0 + c;
  const int ky = col_ok ? (int)(q / H) : 0;
  const int kx = col_ok ? (int)(q - (int64_t)ky * H) : 0;
  const bool fy = ky > g.My / 2;
  const float sy = fy ? -1.f : 1.f;
  const int rec0 = (fy ? g.My - ky : ky) * H + kx;
  const int zrec = g.Oy * H;
  int off[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const int kz = j + r * RA;
    off[r] = (kz > L / 2 ? L - kz : kz) * zrec + rec0;
  }

#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    // potential outputs (half 0: kernels 0..5, Eq. 12 pairs shared) or
    // normal-field outputs (half 1: kernels 6..14, times -i), one output
    // grid at a time; the 3 RB kernel values of a grid are loaded together
    // (the kernel stride passes through an opaque move and the empty asm
    // statements separate the grids, so that the compiler neither hoists
    // the 162 load addresses out of this loop nor one grid's loads into the
    // previous grid's work: both would only cost registers)
    int ot;
    asm volatile("mov.b32 %0, %1;" : "=r"(ot) : "r"(otot));
    if (half == 0) {
      mac_out<0, 0, RA, RB, NT, TX, LD>(spec, ot, off, col_ok, sy, S, t, j, c, ph, buf);
      asm volatile("" ::: "memory");
      mac_out<0, 1, RA, RB, NT, TX, LD>(spec, ot, off, col_ok, sy, S, t, j, c, ph, buf);
      asm volatile("" ::: "memory");
      mac_out<0, 2, RA, RB, NT, TX, LD>(spec, ot, off, col_ok, sy, S, t, j, c, ph, buf);
    } else {
      mac_out<1, 0, RA, RB, NT, TX, LD>(spec, ot, off, col_ok, sy, S, t, j, c, ph, buf);
      asm volatile("" ::: "memory");
      mac_out<1, 1, RA, RB, NT, TX, LD>(spec, ot, off, col_ok, sy, S, t, j, c, ph, buf);
      asm volatile("" ::: "memory");
      mac_out<1, 2, RA, RB, NT, TX, LD>(spec, ot, off, col_ok, sy, S, t, j, c, ph, buf);
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
  const size_t sm = ((size_t)L * 3 * TX + (size_t)3 * RB * RA * TX + pz.twn + pv.twn + L) * sizeof(C);
  const int64_t cols = (int64_t)g.My * g.Hx;
  const int64_t tiles = (cols + TX - 1) / TX;
  VC_CHECK(tiles * B < ((int64_t)1 << 31) && (int64_t)g.Hx * g.Oy * g.Oz * kNumKernels < ((int64_t)1 << 31),
           VOXCAP_ERR_UNSUPPORTED, "grid too large for the compiled z pass");
  auto kern = k_zpass_fast<RA, RB, TX>;
  VC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)(tiles * B), RA * TX, sm, st>>>(g, data, h.spec_f.p, (int)((int64_t)g.Hx * g.Oy * g.Oz), pz.stw,
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
