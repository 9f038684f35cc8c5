// y passes of the products (Eqs. 9-11) on compiled plans: the forward
// transform along y of the x-transformed charge planes (zero rows y >= N_y+1
// are the padding and are not read) and the inverse transform back to the
// N_y+1 rows the panels need, with the half-voxel phase of the y grids.
//
// A CTA transforms TX consecutive lines of the flattened (z, kx) index of
// one grid (128- or 64-byte row segments; a tile may run from the end of one
// z plane into the next, so that no tile is left with a ragged remainder of
// a row): the first stage reads HBM into registers and writes the one
// shared-memory buffer, a middle stage runs in place, and the last stage
// writes HBM from registers.  The padded length is at least twice the
// unpadded one, so the forward first stage reads only the lower half of its
// butterfly inputs and the inverse last stage computes only the outputs
// below L / 2.
//
// k_ypass_pipe is the persistent form: a CTA loops over tiles with two
// line buffers; at the start of a tile it issues the cp.async copies of the
// next tile's rows into the other buffer, so that the HBM reads of one tile
// overlap the transform of the previous one, and every stage runs in place
// on shared memory (the last one writes HBM).  It is also instantiated for
// double2: the y passes of the FP64 products.
#include <algorithm>

#include "fast.cuh"

namespace vc {

namespace {

using fast::C;

template <bool INV, int R1, int R2, int R3, int TX, int NT>
__global__ void __launch_bounds__(NT) k_ypass_fast(Geom g, int G, const C* __restrict__ in, C* __restrict__ out,
                                                   int64_t in_bstride, int64_t out_bstride,
                                                   const C* __restrict__ stw, int twn, int off2, int off3,
                                                   const C* __restrict__ phy) {
  using P = fast::Plan<R1, R2, R3>;
  constexpr int L = P::L;
  static_assert(NT % TX == 0, "a thread keeps one line of the tile in every stage");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tws = buf + L * TX;
  C* phs = tws + twn;                 // half-voxel phases of the y grid
  fast::load_table<NT>(tws, stw, twn);
  fast::load_table<NT>(phs, phy, L);
  const int H = g.Hx;
  const int bg = blockIdx.y;
  const int grid = bg % G, b = bg / G;
  const bool phase = (grid % 3) == 1;
  const int Lin = INV ? L : g.Ly;
  const int Lout = INV ? g.Ly : L;
  // this thread's line: q = z * H + kx
  const int64_t q = (int64_t)blockIdx.x * TX + (int)threadIdx.x % TX;
  const bool ok = q < (int64_t)g.Lz * H;
  const int z = ok ? (int)(q / H) : 0;
  const int kx = ok ? (int)(q - (int64_t)z * H) : 0;
  const C* src = in + (int64_t)b * in_bstride + ((int64_t)grid * g.Lz + z) * ((int64_t)Lin * H) + kx;
  C* dst = out + (int64_t)b * out_bstride + ((int64_t)grid * g.Lz + z) * ((int64_t)Lout * H) + kx;
  __syncthreads();
  // first stage: HBM -> registers -> buffer
  fast::stage<L, R1, 1, TX, NT, INV, INV ? R1 : R1 / 2>(
      tws,
      [&](int, int y) -> C {
        C v = mk<C>(0.f, 0.f);
        if (ok && y < Lin) {
          v = src[(int64_t)y * H];
          if (INV && phase) v = cmul(v, cconj(phs[y]));
        }
        return v;
      },
      [&](int c, int pos, C v) { buf[pos * TX + c] = v; });
  __syncthreads();
  if constexpr (P::NST == 3) fast::stage_inplace<L, R2, R1, TX, NT, INV>(buf, tws + off2);
  // last stage: buffer -> registers -> HBM
  fast::stage<L, P::RL, P::NSL, TX, NT, INV, P::RL, INV ? (P::RL + 1) / 2 : P::RL>(
      tws + (P::NST == 3 ? off3 : off2), [&](int c, int pos) -> C { return buf[pos * TX + c]; },
      [&](int, int y, C v) {
        if (ok && y < Lout) {
          if (!INV && phase) v = cmul(v, phs[y]);
          dst[(int64_t)y * H] = v;
        }
      });
}

template <bool INV, int R1, int R2, int R3, int TX, int NT, typename CT = C>
__global__ void __launch_bounds__(NT) k_ypass_pipe(Geom g, int G, const CT* __restrict__ in, CT* __restrict__ out,
                                                   int64_t in_bstride, int64_t out_bstride,
                                                   const CT* __restrict__ stw, int twn, int off2, int off3,
                                                   const CT* __restrict__ phy, int ntile, int nitems) {
  using P = fast::Plan<R1, R2, R3>;
  constexpr int L = P::L;
  static_assert(NT % TX == 0, "a thread keeps one line of the tile in every stage");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* bufs = reinterpret_cast<CT*>(smem_raw);   // [2][L][TX]
  CT* tws = bufs + 2 * L * TX;
  CT* phs = tws + twn;                          // half-voxel phases of the y grid
  fast::load_table<NT>(tws, stw, twn);
  fast::load_table<NT>(phs, phy, L);
  const int H = g.Hx;
  const int Lin = INV ? L : g.Ly;
  const int Lout = INV ? g.Ly : L;
  const int64_t lines = (int64_t)g.Lz * H;
  const int c = (int)threadIdx.x % TX;           // this thread's line of every tile
  // the global offset of this thread's line in tile `item` (or -1 past the end)
  auto line_of = [&](int item, int64_t bstride, int len, int& grid) -> int64_t {
    const int bg = item / ntile, tile = item - bg * ntile;
    grid = bg % G;
    const int b = bg / G;
    const int64_t q = (int64_t)tile * TX + c;
    if (q >= lines) return -1;
    const int z = (int)(q / H), kx = (int)(q - (int64_t)z * H);
    return (int64_t)b * bstride + ((int64_t)grid * g.Lz + z) * ((int64_t)len * H) + kx;
  };
  auto prefetch = [&](int item, CT* buf) {
    int grid;
    const int64_t o = line_of(item, in_bstride, Lin, grid);
    if (o >= 0) {
      const CT* src = in + o;
      for (int y = (int)threadIdx.x / TX; y < Lin; y += NT / TX)
        fast::cp_async_elem(&buf[y * TX + c], src + (int64_t)y * H);
    }
    fast::cp_async_commit();
  };
  int cur = 0;
  if ((int)blockIdx.x < nitems) prefetch(blockIdx.x, bufs);
  for (int item = blockIdx.x; item < nitems; item += gridDim.x, cur ^= 1) {
    CT* buf = bufs + cur * L * TX;
    fast::cp_async_wait_all();
    __syncthreads();                 // this tile's rows are in; the other buffer is free
    if (item + (int)gridDim.x < nitems) prefetch(item + gridDim.x, bufs + (cur ^ 1) * L * TX);
    int grid;
    const int64_t oo = line_of(item, out_bstride, Lout, grid);
    const bool phase = (grid % 3) == 1;
    // first stage in place: rows >= Lin are the zero padding (the forward
    // pass reads only the lower half of its butterflies' inputs)
    fast::stage_inplace_ld<L, R1, 1, TX, NT, INV, TX, INV ? R1 : R1 / 2>(
        buf, tws, [&](int cc, int y) -> CT {
          CT v = mk<CT>(0, 0);
          if (y < Lin) {
            v = buf[y * TX + cc];
            if (INV && phase) v = cmul(v, cconj(phs[y]));
          }
          return v;
        });
    if constexpr (P::NST == 3) fast::stage_inplace<L, R2, R1, TX, NT, INV>(buf, tws + off2);
    // last stage: buffer -> registers -> HBM
    CT* dst = out + (oo >= 0 ? oo : 0);
    fast::stage<L, P::RL, P::NSL, TX, NT, INV, P::RL, INV ? (P::RL + 1) / 2 : P::RL>(
        tws + (P::NST == 3 ? off3 : off2), [&](int cc, int pos) -> CT { return buf[pos * TX + cc]; },
        [&](int, int y, CT v) {
          if (oo >= 0 && y < Lout) {
            if (!INV && phase) v = cmul(v, phs[y]);
            dst[(int64_t)y * H] = v;
          }
        });
  }
  fast::cp_async_wait_all();
}

template <bool INV, int R1, int R2, int R3, int TX, int NT, typename CT = C>
int launch_ypipe(const Handle& h, int G, const CT* in, CT* out, int64_t ibs, int64_t obs, int B, cudaStream_t st) {
  const Geom& g = h.g;
  constexpr bool F64 = sizeof(CT) == 16;
  const Plan1D<CT>& p = *reinterpret_cast<const Plan1D<CT>*>(F64 ? (const void*)&h.pd[1] : (const void*)&h.pf[1]);
  const CT* phy = reinterpret_cast<const CT*>(F64 ? (const void*)h.phd[1] : (const void*)h.phf[1]);
  constexpr int L = R1 * R2 * R3;
  const size_t sm = ((size_t)2 * L * TX + p.twn + L) * sizeof(CT);
  auto kern = k_ypass_pipe<INV, R1, R2, R3, TX, NT, CT>;
  VC_TRY(set_smem(kern, sm));
  VC_CHECK(2 * g.Ly <= L, VOXCAP_ERR_UNSUPPORTED, "y padding shorter than twice the grid");
  const int64_t ntile = ((int64_t)g.Lz * g.Hx + TX - 1) / TX;
  const int64_t items = ntile * B * G;
  VC_CHECK(items < ((int64_t)1 << 31), VOXCAP_ERR_UNSUPPORTED, "grid too large for the y pass");
  int per_sm = 0, sms = 0;
  VC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm));
  VC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h.device));
  VC_CHECK(per_sm > 0, VOXCAP_ERR_UNSUPPORTED, "the persistent y pass does not fit an SM");
  const int grid = (int)std::min<int64_t>(items, (int64_t)per_sm * sms);
  kern<<<grid, NT, sm, st>>>(g, G, in, out, ibs, obs, p.stw, p.twn, p.twoff[1], p.nst >= 3 ? p.twoff[2] : 0, phy,
                             (int)ntile, (int)items);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

template <bool INV, int R1, int R2, int R3, int TX, int NT>
int launch_y(const Handle& h, int G, const C* in, C* out, int64_t ibs, int64_t obs, int B, cudaStream_t st) {
  const Geom& g = h.g;
  const Plan1D<float2>& p = h.pf[1];
  constexpr int L = R1 * R2 * R3;
  const size_t sm = ((size_t)L * TX + p.twn + L) * sizeof(C);
  auto kern = k_ypass_fast<INV, R1, R2, R3, TX, NT>;
  VC_TRY(set_smem(kern, sm));
  VC_CHECK(2 * g.Ly <= L, VOXCAP_ERR_UNSUPPORTED, "y padding shorter than twice the grid");
  const int64_t tiles = ((int64_t)g.Lz * g.Hx + TX - 1) / TX;
  VC_CHECK(tiles < ((int64_t)1 << 31) && B * G <= 65535, VOXCAP_ERR_UNSUPPORTED, "grid too large for the y pass");
  dim3 grid((unsigned)tiles, B * G);
  kern<<<grid, NT, sm, st>>>(g, G, in, out, ibs, obs, p.stw, p.twn, p.twoff[1], p.nst >= 3 ? p.twoff[2] : 0,
                             h.phf[1]);
  ::vc::note_launch();
  VC_CUDA(cudaGetLastError());
  return VOXCAP_OK;
}

template <bool INV>
int dispatch_y(const Handle& h, int G, const C* in, C* out, int64_t ibs, int64_t obs, int B, int variant,
               cudaStream_t st) {
  const Plan1D<float2>& p = h.pf[1];
  const int* r = p.radix;
  // variant 0: one tile per CTA, the first stage's butterflies at once where
  // that fits in a block; variant 1: the persistent pass (two buffers of
  // 64-byte row segments, or 128-byte ones where they fit)
#define VC_Y(A, B_, C_, TXA, NTA, TXP, NTP)                                         \
  return variant == 1 ? launch_ypipe<INV, A, B_, C_, TXP, NTP>(h, G, in, out, ibs, obs, B, st) \
                      : launch_y<INV, A, B_, C_, TXA, NTA>(h, G, in, out, ibs, obs, B, st)
  if (p.nst == 2) {
    if (r[0] == 4 && r[1] == 9) VC_Y(4, 9, 1, 16, 144, 16, 144);
    if (r[0] == 8 && r[1] == 9) VC_Y(8, 9, 1, 16, 144, 16, 144);
    if (r[0] == 16 && r[1] == 9) VC_Y(16, 9, 1, 16, 144, 16, 144);
  } else if (p.nst == 3 && r[2] == 9) {
    if (r[0] == 8 && r[1] == 4) VC_Y(8, 4, 9, 16, 288, 16, 288);
    if (r[0] == 16 && r[1] == 4) VC_Y(16, 4, 9, 16, 288, 8, 576);
    if (r[0] == 16 && r[1] == 8) VC_Y(16, 8, 9, 16, 576, 8, 576);
  }
#undef VC_Y
  set_error("no compiled y-pass plan for this length");
  return VOXCAP_ERR_UNSUPPORTED;
}

// FP64: the persistent pass, tile widths for about 74 KB per line buffer
template <bool INV>
int dispatch_y64(const Handle& h, int G, const double2* in, double2* out, int64_t ibs, int64_t obs, int B,
                 cudaStream_t st) {
  const Plan1D<double2>& p = h.pd[1];
  const int* r = p.radix;
  using D = double2;
  if (p.nst == 2) {
    if (r[0] == 4 && r[1] == 9) return launch_ypipe<INV, 4, 9, 1, 16, 144, D>(h, G, in, out, ibs, obs, B, st);
    if (r[0] == 8 && r[1] == 9) return launch_ypipe<INV, 8, 9, 1, 16, 144, D>(h, G, in, out, ibs, obs, B, st);
    if (r[0] == 16 && r[1] == 9) return launch_ypipe<INV, 16, 9, 1, 16, 144, D>(h, G, in, out, ibs, obs, B, st);
  } else if (p.nst == 3 && r[2] == 9) {
    if (r[0] == 8 && r[1] == 4) return launch_ypipe<INV, 8, 4, 9, 8, 288, D>(h, G, in, out, ibs, obs, B, st);
    if (r[0] == 16 && r[1] == 4) return launch_ypipe<INV, 16, 4, 9, 4, 144, D>(h, G, in, out, ibs, obs, B, st);
    if (r[0] == 16 && r[1] == 8) return launch_ypipe<INV, 16, 8, 9, 4, 288, D>(h, G, in, out, ibs, obs, B, st);
  }
  set_error("no compiled y-pass plan for this length");
  return VOXCAP_ERR_UNSUPPORTED;
}

}  // namespace

int fast_ypass_f64(const Handle& h, bool inv, int G, const double2* in, double2* out, int64_t in_bstride,
                   int64_t out_bstride, int B, cudaStream_t st) {
  if (inv) return dispatch_y64<true>(h, G, in, out, in_bstride, out_bstride, B, st);
  return dispatch_y64<false>(h, G, in, out, in_bstride, out_bstride, B, st);
}

bool fast_plan_ok(const Plan1D<float2>& p) {
  const int* r = p.radix;
  if (p.nst == 2) return r[1] == 9 && (r[0] == 4 || r[0] == 8 || r[0] == 16);
  if (p.nst == 3) return r[2] == 9 && ((r[0] == 8 && r[1] == 4) || (r[0] == 16 && (r[1] == 4 || r[1] == 8)));
  return false;
}

int fast_ypass(const Handle& h, bool inv, int G, const float2* in, float2* out, int64_t in_bstride,
               int64_t out_bstride, int B, int variant, cudaStream_t st) {
  if (inv) return dispatch_y<true>(h, G, in, out, in_bstride, out_bstride, B, variant, st);
  return dispatch_y<false>(h, G, in, out, in_bstride, out_bstride, B, variant, st);
}

}  // namespace vc
