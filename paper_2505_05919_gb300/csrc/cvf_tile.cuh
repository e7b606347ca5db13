// cvf_tile.cuh -- one tile of the checkerboard sweep (Sec. II.C read for the
// 2D lattice: colour (x + y) & 1, colour 0 first), shared by the
// single-lattice kernel and the batched persistent kernel.
//
// A tile is TR rows x TW 32-bit words (two cells per word, one of each
// colour).  The block stages the tile plus a halo of two rows and one word
// from the step's source buffer, updates the colour-0 cells of the tile and
// of the one-cell ring around it (the ring's updates are recomputed
// identically by the neighbouring tile: same inputs, same counter-based
// draws), then the colour-1 cells of the tile, and writes the tile to the
// step's destination buffer.
#pragma once
#include <cstdint>

#include "cvf_device.cuh"
#include "cvf_tma.cuh"

namespace cvf {

// Shared tables of one (lattice, step): the proposal for the current q and
// the threshold rows of the current gate.
//   prop[8 k + sigma] = {sigma * 0x11111111, ((sigma + 1 + k) mod q) *
//                       0x11111111} for k < 7 (sigma and sigma' in every
//                       nibble; k <= q - 2 <= 6): both words an update needs
//                       in one 8-byte load at byte offset 64 k + 8 sigma
//   rows[9 ps + pp]   = {T - 1, packed count change} for the nibble counts ps,
//                       pp of update_arm2 (entries no move can reach are 0);
//                       an accepted move adds the change (1 << 20) +
//                       ((dN_HB + 1) << 10) + dN_sigma + 3
//   T64[9 ps + pp]    = T (the 64-bit compare, when some T is 0)
constexpr int kRows2 = 72;
struct Tables2 {
  uint2 rows[kRows2];
  uint2 prop[64];
  unsigned long long T64[kRows2];
};

// Proposal part of the tables (depends on q only).
__device__ __forceinline__ void fill_prop2(Tables2& Tb, uint32_t q) {
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    const uint32_t k = (uint32_t)e >> 3, s = (uint32_t)e & 7u;
    uint32_t v = 0u;
    if (s < q && k + 1u < q) {
      uint32_t sp = s + 1u + k;
      while (sp >= q) sp -= q;
      v = sp * 0x11111111u;
    }
    Tb.prop[e] = make_uint2(s * 0x11111111u, v);
  }
}

// Threshold part from a [g][(dN_HB+1)*8 + dN_sigma+3] table of 24 per gate.
// Entry 9 ps + pp: ps = A_s + 4 b_s with A_s <= 3 the arms differing from
// sigma and b_s = [partner != sigma]; pp = A_p + 4 b_p with 1 <= A_p <= 4
// for sigma' -- so b_s = ps >> 2, A_s = ps & 3, b_p = [pp >= 5], A_p = pp -
// 4 b_p, dN_HB = b_s - b_p and dN_sigma = A_s - A_p + 1.
__device__ __forceinline__ void fill_rows2(Tables2& Tb, const unsigned long long* table24, int g) {
  for (int i = threadIdx.x; i < kRows2; i += blockDim.x) {
    const int ps = i / 9, pp = i % 9;
    const int bs = ps >> 2, as = ps & 3, bp = (pp >= 5) ? 1 : 0, ap = pp - 4 * bp;
    if (ap < 1) {  // unreachable: arm a itself always differs from sigma'
      Tb.rows[i] = make_uint2(0u, 0u);
      Tb.T64[i] = 0ull;
      continue;
    }
    const int dhb = bs - bp, dc = as - ap + 1;
    const unsigned long long t = table24[g * 24 + (dhb + 1) * 8 + (dc + 3)];
    Tb.rows[i] = make_uint2((uint32_t)(t - 1ull),  // every t >= 1 unless 64-bit compares
                            (1u << 20) + ((uint32_t)(dhb + 1) << 10) + (uint32_t)(dc + 3));
    Tb.T64[i] = t;
  }
}

constexpr uint32_t kNib1 = 0x11111111u;   // 1 in every nibble
constexpr uint32_t kGuard = 0x88888888u;  // bit 3 of every nibble

// The partner operand of update_arm2 from a partner value pa placed at bits
// 16..18: pa copied into nibbles 4..7 and bit 3 of every nibble set.
__device__ __forceinline__ uint32_t partner_operand(uint32_t pa16) {
  return pa16 * 0x1111u + kGuard;
}

// Metropolis update of arm a of a cell word w (sigma_b in nibble b, b =
// 0..3, nibbles 4..7 zero) with draw u and proposal offset k (Sec. II.C,
// Eq. H).  x is the partner operand: the partner value (arm a^1 of the
// neighbour in direction a) in nibbles 4..7 and bit 3 of every nibble set.
// For v = sigma or sigma' (v R = v in every nibble), t = w ^ v R ^ x holds
// in each nibble 8 + (nibble ^ v), so f(v) = (t - R) & M has bit 3 of nibble
// b set iff nibble b differs from v (no borrow crosses a nibble).  popc f
// (sigma) = A_s + 4 b_s and popc f(sigma') = A_p + 4 b_p index the rows
// directly.  ARM >= 0 fixes a at compile time; ARM = -1 takes it from a_rt.
template <bool CMP64, int ARM = -1>
__device__ __forceinline__ uint32_t update_arm2(uint32_t w, uint32_t x, uint32_t u, uint32_t k,
                                                uint32_t a_rt, const Tables2& Tb, uint32_t& pk) {
  const uint32_t a = (ARM >= 0) ? (uint32_t)ARM : a_rt;
  // 8 sigma: the byte offset of sigma's entry in a proposal table row
  uint32_t s8;
  if constexpr (ARM == 0)
    s8 = (w << 3) & 0x38u;
  else if constexpr (ARM > 0)
    s8 = (w >> (4 * ARM - 3)) & 0x38u;
  else
    s8 = ((w >> (4u * a)) & 7u) << 3;
  const uint2 pr = *reinterpret_cast<const uint2*>(reinterpret_cast<const char*>(Tb.prop) +
                                                   (k << 6) + s8);
  const uint32_t sR = pr.x;   // sigma in every nibble
  const uint32_t spR = pr.y;  // sigma' in every nibble
  const uint32_t fs = ((w ^ sR ^ x) - kNib1) & kGuard;
  const uint32_t fp = ((w ^ spR ^ x) - kNib1) & kGuard;
  const uint32_t idx = (uint32_t)__popc(fs) * 9u + (uint32_t)__popc(fp);
  const uint2 row = Tb.rows[idx];
  const bool accept = CMP64 ? ((unsigned long long)u < Tb.T64[idx]) : (u <= row.x);
  if (accept) {
    const uint32_t mask = 0xFu << (4u * a);
    w = (w & ~mask) | (spR & mask);
    pk += row.y;
  }
  return w;
}

// Count word of a cell: nibble v = number of its arms in state v.
__device__ __forceinline__ uint32_t count_word4(uint32_t w) {
  uint32_t c = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) c += 1u << (4u * ((w >> (4 * b)) & 7u));
  return c;
}

// Philox key material of the lattice being swept: a pointer to its
// precomputed round keys (the tiled sweep's kernel parameter, read from the
// constant bank).
struct KeysRound {
  const RoundKeys* K;
};

template <int RNG_WORDS>
__device__ __forceinline__ void draws(uint32_t c, uint32_t s_lo, uint32_t s_hi, const KeysRound& k,
                                      uint32_t q, uint32_t acc[4], uint32_t kk[4]) {
  cell_draws<RNG_WORDS>(c, s_lo, s_hi, *k.K, q, acc, kk);
}

// The round keys held by value: a copy of a kernel parameter's keys (the
// small lattice resident in one cluster; the compiler takes them from the
// parameter bank as instruction operands).
struct KeysInRegs {
  RoundKeys K;
};

template <int RNG_WORDS>
__device__ __forceinline__ void draws(uint32_t c, uint32_t s_lo, uint32_t s_hi,
                                      const KeysInRegs& k, uint32_t q, uint32_t acc[4],
                                      uint32_t kk[4]) {
  cell_draws<RNG_WORDS>(c, s_lo, s_hi, k.K, q, acc, kk);
}

// The round keys by value and the step's folded first Philox rounds
// (step_draw): the draws take 18 widening multiplies per cell instead of 20
// (the wavefront sweep and the batched kernel, which have the registers for
// the keys: 4096^2 104.7 against 106.7 us per step, 2048^2 32.2 against
// 33.8; the tiled sweep, whose partly filled last round of tiles takes up
// the cycles saved, ran 2 % slower with the folded rounds and keeps
// KeysRound).  The step words passed with it are not used again.
struct KeysStep {
  RoundKeys K;
  StepDraw sd;
};

template <int RNG_WORDS>
__device__ __forceinline__ void draws(uint32_t c, uint32_t, uint32_t, const KeysStep& k,
                                      uint32_t q, uint32_t acc[4], uint32_t kk[4]) {
  cell_draws_step<RNG_WORDS>(c, k.sd, k.K, q, acc, kk);
}

// Update the cell in half `hi` of word `own` (its four arms in order, each
// seeing the earlier ones); xm / xp are the words to the left / right, ym /
// yp the words of the rows y-1 / y+1.  Accepted moves add their packed count
// changes to pk; with s_hist4 (recorded steps) the cell's N_q' is counted.
// HI = 0 / 1 fixes the half at compile time (a warp whose lanes all update
// the same half); HI = -1 takes it from hi_rt.
template <int RNG_WORDS, bool CMP64, int HI = -1, typename KEYS>
__device__ __forceinline__ uint32_t update_in_word(uint32_t own, uint32_t xm_word,
                                                   uint32_t xp_word, uint32_t ym_word,
                                                   uint32_t yp_word, int hi_rt, uint32_t c,
                                                   uint32_t s_lo, uint32_t s_hi,
                                                   const KEYS& keys, uint32_t q,
                                                   const Tables2& Tb, uint32_t& pk,
                                                   uint32_t* s_hist4) {
  // partner operands: arm 0 (+x) <-> arm 1 of the +x cell, arm 1 (-x) <->
  // arm 0 of the -x cell, arm 2 (+y) <-> arm 3 of the +y cell, arm 3 (-y)
  // <-> arm 2 of the -y cell; each partner value, masked where it lies,
  // is copied into nibbles 4..7 by one multiply-add that also sets the
  // guard bits (the multiplier moves it there from its own nibble)
  const int hi = (HI >= 0) ? HI : hi_rt;
  uint32_t w, x0, x1, x2, x3;
  if (hi) {
    w = own >> 16;
    x0 = (xp_word & 0x70u) * 0x1111000u + kGuard;           // nibble 1 of the +x word
    x1 = (own & 0x7u) * 0x11110000u + kGuard;               // nibble 0 of the own word
    x2 = ((yp_word >> 12) & 0x70000u) * 0x1111u + kGuard;   // nibble 7 of the +y word
    x3 = ((ym_word >> 8) & 0x70000u) * 0x1111u + kGuard;    // nibble 6 of the -y word
  } else {
    w = own & 0xFFFFu;
    x0 = ((own >> 4) & 0x70000u) * 0x1111u + kGuard;        // nibble 5 of the own word
    x1 = (xm_word & 0x70000u) * 0x1111u + kGuard;           // nibble 4 of the -x word
    x2 = (yp_word & 0x7000u) * 0x11110u + kGuard;           // nibble 3 of the +y word
    x3 = (ym_word & 0x700u) * 0x111100u + kGuard;           // nibble 2 of the -y word
  }
  uint32_t acc[4], kk[4];
  draws<RNG_WORDS>(c, s_lo, s_hi, keys, q, acc, kk);
  w = update_arm2<CMP64, 0>(w, x0, acc[0], kk[0], 0u, Tb, pk);
  w = update_arm2<CMP64, 1>(w, x1, acc[1], kk[1], 1u, Tb, pk);
  w = update_arm2<CMP64, 2>(w, x2, acc[2], kk[2], 2u, Tb, pk);
  w = update_arm2<CMP64, 3>(w, x3, acc[3], kk[3], 3u, Tb, pk);
  if (s_hist4) hist_add_cell(s_hist4, count_word4(w));
  return hi ? ((own & 0xFFFFu) | (w << 16)) : ((own & 0xFFFF0000u) | w);
}

// Staged input: rows y0-2 .. y0+TR+1 and words p0-4 .. p0+TW+3 (a 16-byte
// aligned box, so one TMA copy can fill it); word p0-1+jj sits in column
// jj+3.  After colour 0: rows y0-1 .. y0+TR, words p0-1 .. p0+TW.
constexpr int kInColOff = 3;
// After colour 0: rows y0-1 .. y0+TR, words p0-1 .. p0+TW, word p0-1+jj in
// column jj+3 as in `in` (rows 16-byte aligned from word p0 on).
constexpr int kMidColOff = 3;
template <int TR, int TW>
struct TileSmem {
  alignas(128) uint32_t in[TR + 4][TW + 8];
  alignas(16) uint32_t mid[TR + 2][TW + 8];
};

// Per-thread totals of the accepted moves of the cells a thread finished
// inside its tiles (ring cells, recomputed by a neighbouring tile that owns
// them, are not counted): their number and the biased sums of dN_HB + 1 and
// dN_sigma + 3, moved out of a phase's packed word after each colour phase
// (a phase adds fewer than 2^10 / 6 moves per thread).
struct TileCounts {
  uint32_t nacc, hb_b, dc_b;
  __device__ __forceinline__ void add(uint32_t pk) {
    nacc += pk >> 20;
    hb_b += (pk >> 10) & 0x3FFu;
    dc_b += pk & 0x3FFu;
  }
  __device__ __forceinline__ int dhb() const { return (int)(hb_b - nacc); }
  __device__ __forceinline__ int dc() const { return (int)(dc_b - 3u * nacc); }
};

// One lattice for one step, as a tile sees it.
template <typename KEYS>
struct StepView {
  const uint32_t* src;  // state words of the step's source buffer
  uint32_t* dst;        // destination buffer
  int L, Lh;
  uint32_t q;
  uint32_t s_lo, s_hi;  // step index
  KEYS keys;
  unsigned int* err;    // error word for the debug build's index checks (or null)
};

// Tile geometry shared by the pieces below.
struct TileGeom {
  int y0, p0, th, tw;
};

template <int TR, int TW>
__device__ __forceinline__ TileGeom tile_geom(int L, int Lh, int y0, int p0) {
  return TileGeom{y0, p0, min(TR, L - y0), min(TW, Lh - p0)};
}

// Stage rows y0-2 .. y0+th+1, words p0-1 .. p0+tw (periodic) with ordinary
// loads (CG: through L2 only -- the source may have been written by other
// SMs since this SM last cached it, without a kernel boundary in between).
template <int TR, int TW, int NT, bool CG, typename KEYS>
__device__ __forceinline__ void stage_plain(const StepView<KEYS>& v, const TileGeom& g,
                                            TileSmem<TR, TW>& S) {
  const int L = v.L, Lh = v.Lh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rr = warp; rr < g.th + 4; rr += NT / 32) {
    int y = g.y0 + rr - 2;
    y = (y < 0) ? y + L : (y >= L ? y - L : y);
    const uint32_t* row = v.src + (size_t)y * Lh;
    for (int jj = lane; jj < g.tw + 2; jj += 32) {
      int p = g.p0 + jj - 1;
      p = (p < 0) ? p + Lh : (p >= Lh ? p - Lh : p);
      if (dcheck(y >= 0 && y < L && p >= 0 && p < Lh && rr < TR + 4 && jj + kInColOff < TW + 8,
                 v.err, kSiteStage))
        S.in[rr][jj + kInColOff] = CG ? __ldcg(row + p) : row[p];
    }
  }
}

// Start the copy of the same rows y0-2 .. y0+th+1 in 16-byte chunks of
// words p0-4 .. p0+tw+3 (columns 0 .. tw+7, so word p0-1 still lands in
// column kInColOff), periodic in chunks, through L2 only.  Needs Lh and p0
// multiples of 4 (every wrapped chunk then starts on a row's 16-byte
// boundary); the caller waits (cp_async_wait_all) and synchronises.
template <int TR, int TW, int NT, typename KEYS>
__device__ __forceinline__ void stage_async16(const StepView<KEYS>& v, const TileGeom& g,
                                              TileSmem<TR, TW>& S) {
  const int L = v.L, Lh = v.Lh;
  const int chunks = (g.tw + 8) >> 2, rows = g.th + 4;
  for (int e = threadIdx.x; e < rows * chunks; e += NT) {
    const int rr = e / chunks, k = e - rr * chunks;
    int y = g.y0 + rr - 2;
    y = (y < 0) ? y + L : (y >= L ? y - L : y);
    int p = g.p0 - 4 + 4 * k;
    p = (p < 0) ? p + Lh : (p >= Lh ? p - Lh : p);
    if (dcheck(y >= 0 && y < L && p >= 0 && p + 4 <= Lh && (p & 3) == 0 && rr < TR + 4 &&
                   4 * k + 4 <= TW + 8,
               v.err, kSiteStage))
      cp_async16_cg(&S.in[rr][4 * k], v.src + (size_t)y * Lh + p);
  }
  cp_async_commit();
}

// Code shape of the colour loops, fixed per kernel at compile time (each
// kernel uses the combination that ran fastest for it):
//   kHalfRows  a warp that covers one row compiles its row loop once per half
//              of the word, so the half a cell occupies is a constant
//   kUnroll0   two cells per loop iteration in colour 0 (two independent arm
//              chains for the scheduler), kUnroll1 the same in colour 1
//   kSplitRec  recorded steps (N_q' counted) run a copy of the row loop of
//              their own, so the other steps test no histogram pointer per
//              cell
enum TileShapeFlags : int { kHalfRows = 1, kUnroll0 = 2, kUnroll1 = 4, kSplitRec = 8 };

// Runs row(half, recorded) with the half and the recorded flag as
// compile-time constants where SHAPE asks for them (-1 / true otherwise).
template <int SHAPE, int ROWS_PER_WARP, typename ROW>
__device__ __forceinline__ void dispatch_row(const ROW& row, int hi, bool recorded) {
  auto halves = [&](auto rec_c) {
    if constexpr (ROWS_PER_WARP == 1 && (SHAPE & kHalfRows) != 0) {
      if (hi)
        row(std::integral_constant<int, 1>{}, rec_c);
      else
        row(std::integral_constant<int, 0>{}, rec_c);
    } else {
      row(std::integral_constant<int, -1>{}, rec_c);
    }
  };
  if constexpr ((SHAPE & kSplitRec) != 0) {
    if (recorded)
      halves(std::true_type{});
    else
      halves(std::false_type{});
  } else {
    halves(std::true_type{});
  }
}

// Colour 0: tile rows -1 .. th, words 0 .. tw-1 (the colour-0 cell of a word
// is its low half on even rows, its high half on odd rows), then the one
// colour-0 cell per row just outside the tile (x0 - 1, high half of word -1,
// on odd rows; x0 + 2 tw, low half of word tw, on even rows).  Reads S.in,
// writes S.mid.  s_hist4 != nullptr (recorded steps): N_q' of the tile's
// cells is counted.
template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, int SHAPE, typename KEYS>
__device__ __forceinline__ void colour0(const StepView<KEYS>& v, const TileGeom& g,
                                        TileSmem<TR, TW>& S, const Tables2& Tb,
                                        TileCounts& cnt, uint32_t* s_hist4) {
  constexpr int kRows = (TW >= 32) ? 1 : 32 / TW;  // rows per warp pass
  constexpr int kLanes = (TW >= 32) ? 32 : TW;     // lanes per row
  constexpr int C = kInColOff + 1;                 // column of word 0
  constexpr int kUnroll = (SHAPE & kUnroll0) ? 2 : 1;
  const int L = v.L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lrow = lane / kLanes, lcol = lane % kLanes;
  const int th = g.th, tw = g.tw, y0 = g.y0, p0 = g.p0;
  uint32_t pk = 0;
  for (int r0 = warp * kRows - 1; r0 <= th; r0 += (NT / 32) * kRows) {
    const int r = r0 + lrow;
    if (r > th) continue;
    const int y = y0 + r;
    const int hi = y & 1;
    const int yg = (y < 0) ? y + L : (y >= L ? y - L : y);
    const bool inside = (r >= 0) && (r < th);
    auto row = [&](auto hi_c, auto rec_c) {
      uint32_t* const hist = decltype(rec_c)::value ? (inside ? s_hist4 : nullptr) : nullptr;
#pragma unroll(kUnroll)
      for (int j = lcol; j < tw; j += kLanes) {
        if (!dcheck(r + 1 >= 0 && r + 3 < TR + 4 && j + C + 1 < TW + 8 && j + C < TW + 8, v.err,
                    kSiteTileRead))
          continue;
        const int xg = 2 * (p0 + j) + hi;
        uint32_t pk_row = 0;
        const uint32_t out = update_in_word<RNG_WORDS, CMP64, decltype(hi_c)::value>(
            S.in[r + 2][j + C], S.in[r + 2][j + C - 1], S.in[r + 2][j + C + 1],
            S.in[r + 1][j + C], S.in[r + 3][j + C], hi, (uint32_t)((long long)yg * L + xg),
            v.s_lo, v.s_hi, v.keys, v.q, Tb, pk_row, hist);
        if (inside) pk += pk_row;  // the halo rows belong to other tiles
        S.mid[r + 1][j + C] = out;
      }
    };
    dispatch_row<SHAPE, kRows>(row, hi, s_hist4 != nullptr);
  }
  cnt.add(pk);
  // the ring goes to the warps after the first two, which take one row of
  // the th + 2 fewer than warps 0 and 1 when 8 warps share 66 rows; with two
  // rows per warp pass (16-word tiles) warp 0 takes the two extra rows, and
  // the ring starts at warp 1
  const int ring0 = (NT >= 128) ? ((TW >= 32) ? 64 : 32) : 0;
  for (int i = (int)threadIdx.x - ring0; i < th + 2; i += NT) {
    if (i < 0) continue;
    const int r = i - 1;
    const int y = y0 + r;
    const int hi = y & 1;
    const int j = hi ? -1 : tw;
    const int yg = (y < 0) ? y + L : (y >= L ? y - L : y);
    int xg = 2 * (p0 + j) + hi;
    xg = (xg < 0) ? xg + L : (xg >= L ? xg - L : xg);
    uint32_t not_counted = 0;  // the ring cells belong to the neighbouring tiles
    // the unused side of the ring word is clamped into the staged columns
    const int jm = max(j, 0), jp = min(j + 2, tw + 1);
    if (!dcheck(r + 1 >= 0 && r + 3 < TR + 4 && j + C >= 0 && j + C < TW + 8 &&
                    jp + kInColOff < TW + 8,
                v.err, kSiteTileRead))
      continue;
    S.mid[r + 1][j + C] = update_in_word<RNG_WORDS, CMP64>(
        S.in[r + 2][j + C], S.in[r + 2][jm + kInColOff], S.in[r + 2][jp + kInColOff],
        S.in[r + 1][j + C], S.in[r + 3][j + C], hi, (uint32_t)((long long)yg * L + xg), v.s_lo,
        v.s_hi, v.keys, v.q, Tb, not_counted, nullptr);
  }
}

// Colour 1: tile rows 0 .. th-1 (low half on odd rows, high on even rows),
// from S.mid to the destination buffer.
template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, int SHAPE, typename KEYS>
__device__ __forceinline__ void colour1(const StepView<KEYS>& v, const TileGeom& g,
                                        TileSmem<TR, TW>& S, const Tables2& Tb,
                                        TileCounts& cnt, uint32_t* s_hist4) {
  constexpr int kRows = (TW >= 32) ? 1 : 32 / TW;
  constexpr int kLanes = (TW >= 32) ? 32 : TW;
  constexpr int kUnroll = (SHAPE & kUnroll1) ? 2 : 1;
  constexpr int M = kMidColOff + 1;  // column of word 0 in S.mid
  const int L = v.L, Lh = v.Lh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lrow = lane / kLanes, lcol = lane % kLanes;
  const int th = g.th, tw = g.tw, y0 = g.y0, p0 = g.p0;
  uint32_t pk = 0;
  for (int r0 = warp * kRows; r0 < th; r0 += (NT / 32) * kRows) {
    const int r = r0 + lrow;
    if (r >= th) continue;
    const int y = y0 + r;
    const int hi = (y & 1) ^ 1;
    uint32_t* drow = v.dst + (size_t)y * Lh + p0;
    auto row = [&](auto hi_c, auto rec_c) {
      uint32_t* const hist = decltype(rec_c)::value ? s_hist4 : nullptr;
#pragma unroll(kUnroll)
      for (int j = lcol; j < tw; j += kLanes) {
        if (!dcheck(r + 2 < TR + 2 && j + M + 1 < TW + 8 && y >= 0 && y < L && p0 + j < Lh, v.err,
                    kSiteTileWrite))
          continue;
        const int xg = 2 * (p0 + j) + hi;
        drow[j] = update_in_word<RNG_WORDS, CMP64, decltype(hi_c)::value>(
            S.mid[r + 1][j + M], S.mid[r + 1][j + M - 1], S.mid[r + 1][j + M + 1],
            S.mid[r][j + M], S.mid[r + 2][j + M], hi, (uint32_t)((long long)y * L + xg), v.s_lo,
            v.s_hi, v.keys, v.q, Tb, pk, hist);
      }
    };
    dispatch_row<SHAPE, kRows>(row, hi, s_hist4 != nullptr);
  }
  cnt.add(pk);
}

// ---------------------------------------------------------------------------
// Full tiles (th = TR, tw = TW, y0 even, Lh a multiple of 4): each thread
// walks down one word column through TR / (NT / TW) consecutive rows, two
// rows per iteration (even row: the colour-0 cell in the low half, odd row:
// in the high half, so both halves are compile-time constants), keeping the
// rows above and below in registers (three shared loads per cell instead of
// five).  Colour 0's halo rows -1 and TR and its ring of single cells follow
// as one cell per thread.  Colour 1 writes each word back in place (a
// colour-1 update reads only the colour-0 halves of its neighbours, which
// colour 1 does not change), and the tile is copied out with 16-byte loads
// and stores.  PAIRS: row pairs per loop iteration (the compiler's unroll
// factor; 2 where the kernel has the registers for it: the wavefront sweep
// at 64 registers, 4096^2 103.0 against 104.8 us per step; the tiled sweep at
// 48 registers keeps 1, where 2 spilled 76 bytes and ran at 563 against 583
// sigma-updates/ns).
// ---------------------------------------------------------------------------
template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, bool REC, int PAIRS,
          typename KEYS>
__device__ __forceinline__ void colour0_walk(const StepView<KEYS>& v, const TileGeom& g,
                                             TileSmem<TR, TW>& S, const Tables2& Tb,
                                             TileCounts& cnt, uint32_t* s_hist4) {
  constexpr int kGroups = NT / TW, kRows = TR / kGroups;
  static_assert(NT % TW == 0 && TR % kGroups == 0 && kRows % 2 == 0, "walk shape");
  constexpr int C = kInColOff + 1;  // column of word 0 (S.in and S.mid)
  constexpr int P = TW + 8;         // row pitch (words) of S.in and S.mid
  const uint32_t L = (uint32_t)v.L;
  const int j = (int)threadIdx.x % TW, r0 = ((int)threadIdx.x / TW) * kRows;
  uint32_t* const hist = REC ? s_hist4 : nullptr;
  {
    const uint32_t* p = &S.in[r0 + 2][j + C];  // own word of row r0
    uint32_t* o = &S.mid[r0 + 1][j + C];
    uint32_t cb = (uint32_t)(g.y0 + r0) * L + 2u * (uint32_t)(g.p0 + j);
    uint32_t ym = p[-P], own = p[0];
    uint32_t pk = 0;
#pragma unroll PAIRS
    for (int k = 0; k < kRows; k += 2) {
      const uint32_t yp = p[P];
      o[0] = update_in_word<RNG_WORDS, CMP64, 0>(own, p[-1], p[1], ym, yp, 0, cb, v.s_lo,
                                                 v.s_hi, v.keys, v.q, Tb, pk, hist);
      const uint32_t yp2 = p[2 * P];
      o[P] = update_in_word<RNG_WORDS, CMP64, 1>(yp, p[P - 1], p[P + 1], own, yp2, 1, cb + L + 1u,
                                                 v.s_lo, v.s_hi, v.keys, v.q, Tb, pk, hist);
      ym = yp;
      own = yp2;
      cb += 2u * L;
      p += 2 * P;
      o += 2 * P;
    }
    cnt.add(pk);
  }
  // rows -1 and TR (other tiles' cells: not counted), then the ring
  const int th = g.th, tw = g.tw, y0 = g.y0, p0 = g.p0;
  for (int i = (int)threadIdx.x; i < 2 * TW + TR + 2; i += NT) {
    int r, jj;
    if (i < 2 * TW) {
      r = (i < TW) ? -1 : TR;
      jj = i % TW;
    } else {
      r = i - 2 * TW - 1;
      jj = ((y0 + r) & 1) ? -1 : tw;
    }
    const int y = y0 + r;
    const int hi = y & 1;
    const int yg = (y < 0) ? y + (int)L : (y >= (int)L ? y - (int)L : y);
    int xg = 2 * (p0 + jj) + hi;
    xg = (xg < 0) ? xg + (int)L : (xg >= (int)L ? xg - (int)L : xg);
    const int jm = max(jj, 0), jp = min(jj + 2, tw + 1);
    uint32_t not_counted = 0;
    if (!dcheck(r + 1 >= 0 && r + 3 < TR + 4 && jj + C >= 0 && jj + C < TW + 8 &&
                    jp + kInColOff < TW + 8 && th == TR,
                v.err, kSiteTileRead))
      continue;
    S.mid[r + 1][jj + C] = update_in_word<RNG_WORDS, CMP64>(
        S.in[r + 2][jj + C], S.in[r + 2][jm + kInColOff], S.in[r + 2][jp + kInColOff],
        S.in[r + 1][jj + C], S.in[r + 3][jj + C], hi, (uint32_t)yg * L + (uint32_t)xg, v.s_lo,
        v.s_hi, v.keys, v.q, Tb, not_counted, nullptr);
  }
}

template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, bool REC, int PAIRS,
          typename KEYS>
__device__ __forceinline__ void colour1_walk(const StepView<KEYS>& v, const TileGeom& g,
                                             TileSmem<TR, TW>& S, const Tables2& Tb,
                                             TileCounts& cnt, uint32_t* s_hist4) {
  constexpr int kGroups = NT / TW, kRows = TR / kGroups;
  constexpr int C = kMidColOff + 1;
  constexpr int P = TW + 8;
  const uint32_t L = (uint32_t)v.L;
  const int j = (int)threadIdx.x % TW, r0 = ((int)threadIdx.x / TW) * kRows;
  uint32_t* const hist = REC ? s_hist4 : nullptr;
  uint32_t* q = &S.mid[r0 + 1][j + C];  // own word of row r0
  uint32_t cb = (uint32_t)(g.y0 + r0) * L + 2u * (uint32_t)(g.p0 + j);
  uint32_t ym = q[-P], own = q[0];
  uint32_t pk = 0;
#pragma unroll PAIRS
  for (int k = 0; k < kRows; k += 2) {
    // even row: the colour-1 cell in the high half; odd row: the low half
    const uint32_t yp = q[P];
    const uint32_t w0 = update_in_word<RNG_WORDS, CMP64, 1>(own, q[-1], q[1], ym, yp, 1, cb + 1u,
                                                            v.s_lo, v.s_hi, v.keys, v.q, Tb, pk,
                                                            hist);
    const uint32_t yp2 = q[2 * P];
    const uint32_t w1 = update_in_word<RNG_WORDS, CMP64, 0>(yp, q[P - 1], q[P + 1], own, yp2, 0,
                                                            cb + L, v.s_lo, v.s_hi, v.keys, v.q,
                                                            Tb, pk, hist);
    reinterpret_cast<uint16_t*>(q)[1] = (uint16_t)(w0 >> 16);
    reinterpret_cast<uint16_t*>(q + P)[0] = (uint16_t)w1;
    ym = yp;
    own = yp2;
    cb += 2u * L;
    q += 2 * P;
  }
  cnt.add(pk);
  __syncthreads();
  // the tile's TR x TW words to the destination, 16 bytes at a time
  constexpr int kVec = TW / 4;
  const size_t Lh = (size_t)v.Lh;
  for (int e = (int)threadIdx.x; e < TR * kVec; e += NT) {
    const int r = e / kVec, c4 = e % kVec;
    const uint4 val = *reinterpret_cast<const uint4*>(&S.mid[r + 1][C + 4 * c4]);
    *reinterpret_cast<uint4*>(v.dst + (size_t)(g.y0 + r) * Lh + (size_t)(g.p0 + 4 * c4)) = val;
  }
}

}  // namespace cvf
