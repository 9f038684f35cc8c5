// z pass of the forward FP32 product (Eqs. 9-12) on compiled two-stage
// plans Mz = RA * RB: forward z transforms of the three charge spectra, the
// spectral multiply-accumulate with the 15 real kernel spectra (6 potential,
// 9 normal-field blocks; Eq. 12 folds the other three potential blocks) and
// the inverse z transforms back to the N_z+1 planes the panels need.
//
// A CTA (RA * TX threads) takes TX consecutive kx columns of one row ky of
// one batch item, the rows taken in the order 0, 1, My-1, 2, My-2, ... so
// that the two rows that share a folded row of the kernel spectra (ky and
// My-ky) run back to back and the second reads the spectra from L2.  The
// FP32 spectra are read in their blocked layout [Oy][Hx/8][Oz][15][8]: the
// spectra of a tile are one or two contiguous blocks of 35 KB (Mz = 144), not
// 1095 rows scattered over the whole octant array.  Stage A (radix RA,
// only its lower RA/2 inputs: planes z >= Mz/2 are padding) reads the N_z+1
// non-zero planes of the three input grids from HBM and fills the shared
// buffer [Mz][3][TX]; each thread
// then holds the RB frequencies kz = j + RA r of its column for all three
// grids (last forward stage, parked in a second shared buffer), multiplies
// them with the real kernel spectra and runs the first inverse stage;
// the outputs go through the first buffer in two halves (potential grids,
// then field grids) to the last inverse stage (radix RA), which writes
// planes z <= N_z to HBM (only the outputs below Mz/2 are computed).
//
// k_zpass_pipe (Mz = 16 * 9, TX = 8) is the persistent form of the same
// pass: a CTA takes tiles from a device counter (in order, so that the tiles
// in flight stay close together and the mirrored rows still share the
// spectra in L2), and while it works on one tile the next tile's input
// planes arrive in a staging buffer by cp.async, so that stage A reads
// shared memory instead of waiting on HBM.  Each thread keeps
// its 27 charge spectra in registers (no second buffer: three CTAs fit an
// SM), loads the kernel values of the next output grid while it computes
// the current one, and folds the fold signs of Eq. 12's real spectra into
// the charge and result spectra: with s_y, s_z = -1 on the mirrored half of
// the y or z frequencies and s_x = 1, the sign of potential block P^{ab} is
// s_a s_b and that of field block E^{ab} is s_b, so the sources are scaled
// by s_b once and the potential results by s_a.
#include <algorithm>

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
__device__ __forceinline__ void mac_out(const float* __restrict__ spec, const int* off, float sy, const C* S,
                                        int t, int j, int c, const C* ph, C* buf) {
  constexpr int L = RA * RB;
  constexpr int K0 = kidx(HALF, AL, 0), K1 = kidx(HALF, AL, 1), K2 = kidx(HALF, AL, 2);
  float kv[RB][3];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    kv[r][0] = __ldg(spec + off[r] + K0 * kSpecBlk);
    kv[r][1] = __ldg(spec + off[r] + K1 * kSpecBlk);
    kv[r][2] = __ldg(spec + off[r] + K2 * kSpecBlk);
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

// Row i of the processing order: 0, 1, My-1, 2, My-2, ..., My/2 (My even).
__device__ __forceinline__ int row_of(int i, int My) {
  const int p = (i + 1) >> 1;
  return (i & 1) || i == 0 ? p : My - p;
}

// offset of column kxa's spectra block entry (kz folded, ky folded) in the
// blocked spectra, without the kernel's K * kSpecBlk
__device__ __forceinline__ int spec_block(const Geom& g, int nm, int kyf, int kxa) {
  return ((kyf * nm + kxa / kSpecBlk) * g.Oz) * (kNumKernels * kSpecBlk) + kxa % kSpecBlk;
}

template <int RA, int RB, int TX>
__global__ void __launch_bounds__(RA * TX, 2) k_zpass_fast(Geom g, C* __restrict__ data,
                                                          const float* __restrict__ spec, int nm,
                                                          const C* __restrict__ twf, int twn_f, int offB,
                                                          const C* __restrict__ twv, int twn_v, int offA_tw,
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
  const int64_t gstride = (int64_t)g.Lz * zstride;
  // the tile: row i of the processing order, columns kx0 .. kx0 + ncol - 1
  const int ntr = (H + TX - 1) / TX;
  const int tile = blockIdx.x / nbatch, i = tile / ntr;
  const int kx0 = (tile - i * ntr) * TX;
  const int ky = row_of(i, g.My);
  const int ncol = min(TX, H - kx0);
  const int col0 = ky * H + kx0;                          // < My H < 2^31 (checked at launch)
  C* base = data + (int64_t)b * 6 * gstride + col0;
  const int Lz = g.Lz;
  __syncthreads();

  // ---- stage A: forward radix RA of the three input grids, HBM -> buffer
  fast::stage<L, RA, 1, LD, NT, false, RA / 2>(
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

  // the column's frequencies (kz folded, ky folded, kx) in the blocked
  // spectra; 32-bit (the launch checks the size); a column past the row's
  // end reads column kx0's values, computed and never stored
  const bool fy = ky > g.My / 2;
  const float sy = fy ? -1.f : 1.f;
  const int sb = spec_block(g, nm, fy ? g.My - ky : ky, kx0 + (c < ncol ? c : 0));
  int off[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const int kz = j + r * RA;
    off[r] = (kz > L / 2 ? L - kz : kz) * (kNumKernels * kSpecBlk) + sb;
  }

#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    // potential outputs (half 0: kernels 0..5, Eq. 12 pairs shared) or
    // normal-field outputs (half 1: kernels 6..14, times -i), one output
    // grid at a time; the 3 RB kernel values of a grid are loaded together
    // (the spectra pointer passes through an opaque move per grid, so that
    // the compiler hoists no grid's loads into the previous grid's work,
    // which would only cost registers)
    const float* sp;
    asm volatile("mov.b64 %0, %1;" : "=l"(sp) : "l"(spec));
    if (half == 0) {
      mac_out<0, 0, RA, RB, NT, TX, LD>(sp, off, sy, S, t, j, c, ph, buf);
      asm volatile("mov.b64 %0, %1;" : "=l"(sp) : "l"(spec));
      mac_out<0, 1, RA, RB, NT, TX, LD>(sp, off, sy, S, t, j, c, ph, buf);
      asm volatile("mov.b64 %0, %1;" : "=l"(sp) : "l"(spec));
      mac_out<0, 2, RA, RB, NT, TX, LD>(sp, off, sy, S, t, j, c, ph, buf);
    } else {
      mac_out<1, 0, RA, RB, NT, TX, LD>(sp, off, sy, S, t, j, c, ph, buf);
      asm volatile("mov.b64 %0, %1;" : "=l"(sp) : "l"(spec));
      mac_out<1, 1, RA, RB, NT, TX, LD>(sp, off, sy, S, t, j, c, ph, buf);
      asm volatile("mov.b64 %0, %1;" : "=l"(sp) : "l"(spec));
      mac_out<1, 2, RA, RB, NT, TX, LD>(sp, off, sy, S, t, j, c, ph, buf);
    }
    __syncthreads();
    // ---- last inverse stage (radix RA), buffer -> HBM, planes z < Lz
    fast::stage<L, RA, RB, LD, NT, true, RA, RA / 2>(
        tv + offA_tw, [&](int line, int pos) -> C { return buf[pos * LD + line]; },
        [&](int line, int z, C v) {
          const int grid = line / TX + 3 * half, cc = line % TX;
          if (cc < ncol && z < Lz) base[grid * gstride + z * zstride + cc] = v;
        });
    __syncthreads();
  }
}

using fast::cp_async8;
using fast::cp_async_commit;
using fast::cp_async_wait_all;

// the RB x 3 kernel values of output grid AL of half HALF at the thread's frequencies
// (the spectra pointer passes through an opaque move, so that the
// compiler issues these 27 loads here rather than all 162 of a tile up front)
template <int HALF, int AL, int RB>
__device__ __forceinline__ void load_kv(const float* __restrict__ spec, const int* off, float (&kv)[RB][3]) {
  constexpr int K0 = kidx(HALF, AL, 0), K1 = kidx(HALF, AL, 1), K2 = kidx(HALF, AL, 2);
  const float* sp;
  asm volatile("mov.b64 %0, %1;" : "=l"(sp) : "l"(spec));
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    kv[r][0] = __ldg(sp + off[r] + K0 * kSpecBlk);
    kv[r][1] = __ldg(sp + off[r] + K1 * kSpecBlk);
    kv[r][2] = __ldg(sp + off[r] + K2 * kSpecBlk);
  }
}

// output grid AL of half HALF from the sign-scaled sources S: the sum over
// the three sources, -i for the field blocks, s_a of the potential blocks
// (s_y, or s_z inside the signed phase table phs), the output phase of z
// grids, the first inverse stage (radix RB), and the store to the buffer
template <int HALF, int AL, int RA, int RB, int TX, int LD>
__device__ __forceinline__ void mac_store(const float (&kv)[RB][3], const C (&S)[3][RB], float sy, int j, int c,
                                          const C* ph, const C* phs, C* buf) {
  C o[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    C acc;
    acc.x = fmaf(S[0][r].x, kv[r][0], fmaf(S[1][r].x, kv[r][1], S[2][r].x * kv[r][2]));
    acc.y = fmaf(S[0][r].y, kv[r][0], fmaf(S[1][r].y, kv[r][1], S[2][r].y * kv[r][2]));
    o[r] = HALF == 0 ? acc : cmul_mi(acc);
    if (HALF == 0 && AL == 1) o[r] = cscale(o[r], sy);
    if (AL == 2) o[r] = cmul(o[r], cconj(HALF == 0 ? phs[j + r * RA] : ph[j + r * RA]));
  }
  dft<RB, C>(o, true);
#pragma unroll
  for (int r = 0; r < RB; ++r) buf[(j * RB + r) * LD + AL * TX + c] = o[r];
}

// the 6 distinct potential kernels (0..5) at the thread's frequencies
template <int RB>
__device__ __forceinline__ void load_pot(const float* __restrict__ spec, const int* off, float (&kp)[6][RB]) {
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int r = 0; r < RB; ++r) kp[k][r] = __ldg(spec + off[r] + k * kSpecBlk);
}

// potential output grid AL from the 6 loaded potential kernels
template <int AL, int RA, int RB, int TX, int LD>
__device__ __forceinline__ void mac_store_pot(const float (&kp)[6][RB], const C (&S)[3][RB], float sy, int j, int c,
                                              const C* ph, const C* phs, C* buf) {
  constexpr int K0 = kidx(0, AL, 0), K1 = kidx(0, AL, 1), K2 = kidx(0, AL, 2);
  float kv[RB][3];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    kv[r][0] = kp[K0][r];
    kv[r][1] = kp[K1][r];
    kv[r][2] = kp[K2][r];
  }
  mac_store<0, AL, RA, RB, TX, LD>(kv, S, sy, j, c, ph, phs, buf);
}

template <int RA, int RB, int TX>
__global__ void __launch_bounds__(RA * TX, 3) k_zpass_pipe(Geom g, C* __restrict__ data,
                                                          const float* __restrict__ spec, int nm,
                                                          const C* __restrict__ twf, int twn_f, int offB,
                                                          const C* __restrict__ twv, int twn_v, int offA_tw,
                                                          const C* __restrict__ phz, int nbatch, int nitems,
                                                          int* __restrict__ queue) {
  constexpr int L = RA * RB, NT = RA * TX, LD = 3 * TX, LH = L / 2;
  __shared__ int s_item[2];                     // tiles taken from the counter, by parity
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);      // [L][3][TX]: z lines between the stages
  C* stg = buf + L * LD;                        // [3][L/2][TX]: the next tile's input planes
  C* tf = stg + 3 * LH * TX;
  C* tv = tf + twn_f;
  C* ph = tv + twn_v;                           // e^{+i pi kz / Mz}
  C* phs = ph + L;                              // s_z(kz) e^{+i pi kz / Mz}
  fast::load_table<NT>(tf, twf, twn_f);
  fast::load_table<NT>(tv, twv, twn_v);
  for (int i = threadIdx.x; i < L; i += NT) {
    const C p = phz[i];
    ph[i] = p;
    phs[i] = i > L / 2 ? mk<C>(-p.x, -p.y) : p;
  }
  const int H = g.Hx, Lz = g.Lz;
  const int64_t zstride = (int64_t)g.My * H;    // one z plane [My][H]
  const int64_t gstride = (int64_t)Lz * zstride;
  const int t = threadIdx.x, j = t / TX, c = t % TX;
  const int ntr = (H + TX - 1) / TX;            // tiles per row
  // tile `item`: batch item b, row ky (row i of the processing order),
  // columns kx0 .. kx0 + ncol - 1 starting at col0 = ky H + kx0 of a plane
  struct Tile {
    int b, ky, kx0, ncol, col0;
  };
  auto tile_of = [&](int item) {
    Tile u;
    u.b = item % nbatch;
    const int tile = item / nbatch, i = tile / ntr;
    u.kx0 = (tile - i * ntr) * TX;
    u.ky = row_of(i, g.My);
    u.ncol = min(TX, H - u.kx0);
    u.col0 = u.ky * H + u.kx0;                  // < My H < 2^31 (checked at launch)
    return u;
  };
  // the input planes of a tile into the staging buffer (asynchronous;
  // thread t copies column t % TX)
  auto prefetch = [&](int item) {
    const Tile u = tile_of(item);
    if (c < u.ncol) {
      const C* src = data + (int64_t)u.b * 6 * gstride + u.col0 + c;
#pragma unroll
      for (int grid = 0; grid < 3; ++grid)
        for (int z = j; z < Lz; z += NT / TX)
          cp_async8(&stg[(grid * LH + z) * TX + c], src + grid * gstride + z * zstride);
    }
    cp_async_commit();
  };

  int par = 0;
  if (t == 0) s_item[0] = atomicAdd(queue, 1);
  __syncthreads();
  int item = s_item[0];
  if (item < nitems) prefetch(item);
  while (item < nitems) {
    // the tile after this one (read by all threads after the barriers below;
    // the slot was last read in the previous tile)
    if (t == 0) s_item[par ^ 1] = atomicAdd(queue, 1);
    const Tile u = tile_of(item);
    const int ncol = u.ncol;
    C* base = data + (int64_t)u.b * 6 * gstride + u.col0;
    cp_async_wait_all();
    __syncthreads();                            // staging and columns of this tile in; buffer free

    // ---- stage A: forward radix RA (lower RA/2 inputs), staging -> buffer
    fast::stage<L, RA, 1, LD, NT, false, RA / 2>(
        tf,
        [&](int line, int z) -> C {
          const int grid = line / TX, cc = line % TX;
          C v = mk<C>(0.f, 0.f);
          if (cc < ncol && z < Lz) v = stg[(grid * LH + z) * TX + cc];
          return v;
        },
        [&](int line, int pos, C v) { buf[pos * LD + line] = v; });
    __syncthreads();                            // buffer complete, staging free
    const int next = s_item[par ^ 1];
    if (next < nitems) prefetch(next);

    // blocked-spectra offsets of the thread's frequencies (kz folded, ky
    // folded, kx; a column past the row's end reads column kx0's values,
    // computed and never stored); the 6 potential kernels are loaded now,
    // ahead of the stage below
    const bool fy = u.ky > g.My / 2;
    const float sy = fy ? -1.f : 1.f;
    const int sb = spec_block(g, nm, fy ? g.My - u.ky : u.ky, u.kx0 + (c < ncol ? c : 0));
    int off[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int kz = j + r * RA;
      off[r] = (kz > L / 2 ? L - kz : kz) * (kNumKernels * kSpecBlk) + sb;
    }
    float kp[6][RB];
    load_pot<RB>(spec, off, kp);
    // ---- last forward stage (radix RB) into registers, sources scaled by s_b
    C S[3][RB];
#pragma unroll
    for (int be = 0; be < 3; ++be) {
      C v[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) v[r] = buf[(j + r * RA) * LD + be * TX + c];
      fast::twiddle<RB, false>(v, tf + offB, j);
      dft<RB, C>(v, false);
#pragma unroll
      for (int r = 0; r < RB; ++r)
        S[be][r] = be == 0 ? v[r] : be == 1 ? cscale(v[r], sy) : cmul(v[r], phs[j + r * RA]);
    }
    __syncthreads();                            // every stage-B input read: the buffer takes the outputs

    // last inverse stage (radix RA with twiddles, outputs below Mz/2) of
    // output grids 3 h .. 3 h + 2, buffer -> HBM, one butterfly at a time
    // (the sources S stay live in registers meanwhile)
    auto last_stage = [&](int h) {
      constexpr int NB = L / RA, TOT = NB * LD;   // butterflies (j', line); NB = RB
#pragma unroll 1
      for (int item = t; item < TOT; item += NT) {
        const int line = item % LD, jj = item / LD;
        C v[RA];
#pragma unroll
        for (int r = 0; r < RA; ++r) v[r] = buf[(jj + r * NB) * LD + line];
        fast::twiddle<RA, true>(v, tv + offA_tw, jj);
        dft<RA, C>(v, true);
        const int grid = line / TX + 3 * h, cc = line % TX;
        if (cc < ncol) {
          C* o = base + grid * gstride + cc + jj * zstride;
#pragma unroll
          for (int r = 0; r < RA / 2; ++r)
            if (jj + r * NB < Lz) o[(int64_t)r * NB * zstride] = v[r];
        }
      }
    };
    // ---- potential outputs
    mac_store_pot<0, RA, RB, TX, LD>(kp, S, sy, j, c, ph, phs, buf);
    mac_store_pot<1, RA, RB, TX, LD>(kp, S, sy, j, c, ph, phs, buf);
    mac_store_pot<2, RA, RB, TX, LD>(kp, S, sy, j, c, ph, phs, buf);
    __syncthreads();
    last_stage(0);
    float ka[RB][3], kb[RB][3];
    load_kv<1, 0, RB>(spec, off, ka);
    __syncthreads();                            // the buffer takes the field outputs
    // ---- field outputs; kernel values loaded one grid ahead
    load_kv<1, 1, RB>(spec, off, kb);
    mac_store<1, 0, RA, RB, TX, LD>(ka, S, sy, j, c, ph, phs, buf);
    load_kv<1, 2, RB>(spec, off, ka);
    mac_store<1, 1, RA, RB, TX, LD>(kb, S, sy, j, c, ph, phs, buf);
    mac_store<1, 2, RA, RB, TX, LD>(ka, S, sy, j, c, ph, phs, buf);
    __syncthreads();
    last_stage(1);
    item = next;
    par ^= 1;
  }
  cp_async_wait_all();
}

template <int RA, int RB, int TX>
int launch_zpipe(const Handle& h, C* data, int B, cudaStream_t st) {
  const Geom& g = h.g;
  const Plan1D<float2>& pz = h.pzf[0];
  const Plan1D<float2>& pv = h.pzfr[0];
  constexpr int L = RA * RB, NT = RA * TX;
  const size_t sm = ((size_t)L * 3 * TX + (size_t)3 * (L / 2) * TX + pz.twn + pv.twn + 2 * L) * sizeof(C);
  const int nm = (g.Hx + kSpecBlk - 1) / kSpecBlk;
  const int64_t items = (int64_t)g.My * ((g.Hx + TX - 1) / TX) * B;
  VC_CHECK(items < ((int64_t)1 << 31) && (int64_t)g.My * g.Hx < ((int64_t)1 << 31) &&
               (int64_t)g.Oy * nm * g.Oz * kNumKernels * kSpecBlk < ((int64_t)1 << 31),
           VOXCAP_ERR_UNSUPPORTED, "grid too large for the compiled z pass");
  VC_CHECK(h.spec_fb.p != nullptr && TX % kSpecBlk == 0, VOXCAP_ERR_UNSUPPORTED, "blocked spectra missing");
  VC_CHECK(2 * g.Lz <= L && g.My % 2 == 0, VOXCAP_ERR_UNSUPPORTED, "z padding shorter than twice the grid or odd My");
  auto kern = k_zpass_pipe<RA, RB, TX>;
  VC_TRY(set_smem(kern, sm));
  int per_sm = 0, sms = 0;
  VC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm));
  VC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h.device));
  VC_CHECK(per_sm > 0, VOXCAP_ERR_UNSUPPORTED, "the persistent z pass does not fit an SM");
  const int grid = (int)std::min<int64_t>(items, (int64_t)per_sm * sms);
  VC_CHECK(h.zqueue.p != nullptr, VOXCAP_ERR_UNSUPPORTED, "tile counter of the persistent z pass missing");
  VC_CUDA(cudaMemsetAsync(h.zqueue.p, 0, sizeof(int), st));
  kern<<<grid, NT, sm, st>>>(g, data, h.spec_fb.p, nm, pz.stw, pz.twn, pz.twoff[1], pv.stw, pv.twn,
                             pv.twoff[1], h.phf[2], B, (int)items, h.zqueue.p);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

template <int RA, int RB, int TX>
int launch_z(const Handle& h, C* data, int B, cudaStream_t st) {
  const Geom& g = h.g;
  const Plan1D<float2>& pz = h.pzf[0];
  const Plan1D<float2>& pv = h.pzfr[0];
  constexpr int L = RA * RB;
  const size_t sm = ((size_t)L * 3 * TX + (size_t)3 * RB * RA * TX + pz.twn + pv.twn + L) * sizeof(C);
  const int nm = (g.Hx + kSpecBlk - 1) / kSpecBlk;
  const int64_t tiles = (int64_t)g.My * ((g.Hx + TX - 1) / TX);
  VC_CHECK(tiles * B < ((int64_t)1 << 31) && (int64_t)g.My * g.Hx < ((int64_t)1 << 31) &&
               (int64_t)g.Oy * nm * g.Oz * kNumKernels * kSpecBlk < ((int64_t)1 << 31),
           VOXCAP_ERR_UNSUPPORTED, "grid too large for the compiled z pass");
  VC_CHECK(2 * g.Lz <= L && g.My % 2 == 0, VOXCAP_ERR_UNSUPPORTED, "z padding shorter than twice the grid or odd My");
  VC_CHECK(h.spec_fb.p != nullptr && TX % kSpecBlk == 0, VOXCAP_ERR_UNSUPPORTED, "blocked spectra missing");
  auto kern = k_zpass_fast<RA, RB, TX>;
  VC_TRY(set_smem(kern, sm));
  kern<<<(unsigned)(tiles * B), RA * TX, sm, st>>>(g, data, h.spec_fb.p, nm, pz.stw, pz.twn, pz.twoff[1], pv.stw,
                                                   pv.twn, pv.twoff[1], h.phf[2], B);
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
    if (p.radix[0] == 16 && h.zfvar == 1) return launch_zpipe<16, 9, 8>(h, data, B, st);
    if (p.radix[0] == 16) return launch_z<16, 9, 16>(h, data, B, st);
    if (p.radix[0] == 8) return launch_z<8, 9, 16>(h, data, B, st);
    if (p.radix[0] == 4) return launch_z<4, 9, 16>(h, data, B, st);
  }
  set_error("no compiled z-pass plan for this length");
  return VOXCAP_ERR_UNSUPPORTED;
}

}  // namespace vc
