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

namespace cvf {

// Proposal lookup for the current q: entry 8 sigma + k holds, for the
// proposed value sigma' = (sigma + 1 + k) mod q, the word 4 sigma', 2^(28 -
// 4 sigma') and 2^(4 sigma') (see update_arms).  Filled by the block.
struct ProposalTable {
  uint32_t t4[64];
  uint32_t m[64];
  uint32_t oh[64];
};

__device__ __forceinline__ void fill_proposal_table(ProposalTable& P, uint32_t q) {
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    const uint32_t s = (uint32_t)e >> 3, k = (uint32_t)e & 7u;
    const uint32_t sp = (s + 1u + k) % q;
    P.t4[e] = 4u * sp;
    P.m[e] = 0x10000000u >> (4u * sp);
    P.oh[e] = 1u << (4u * sp);
  }
}

__device__ __forceinline__ uint32_t lds_at(const uint32_t* base, uint32_t byte_off) {
  return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(base) + byte_off);
}

// Metropolis update of the four arms of one cell, with the count-nibble
// bookkeeping of update_arms (cvf_device.cuh) and the proposal taken from
// the block's ProposalTable.  t4[a] = 4 sigma_a (in/out), nb8[a] = 8 oh(n_a).
template <bool CMP64, bool BONDS>
__device__ __forceinline__ uint32_t update_arms_tab(uint32_t t4[4], const uint32_t nb8[4],
                                                    const uint32_t acc[4], const uint32_t kk[4],
                                                    const ProposalTable& P,
                                                    const typename ThresholdRow<CMP64>::type* T,
                                                    uint32_t& naccepted, uint32_t& pair_sum,
                                                    uint32_t& cnt_out, bool count_pairs) {
  uint32_t oh[4], m[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    oh[a] = 1u << t4[a];
    m[a] = 0x10000000u >> t4[a];
  }
  uint32_t cnt = oh[0] + oh[1] + oh[2] + oh[3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const uint32_t wa = cnt + nb8[a];
    const uint32_t off = 8u * t4[a] + 4u * kk[a];  // byte offset of entry 8 sigma + k
    const uint32_t tp = lds_at(P.t4, off);
    const uint32_t mp = lds_at(P.m, off);
    const uint32_t ohp = lds_at(P.oh, off);
    const int fsp = (int)nibble(wa, mp);
    const int fs = (int)nibble(wa, m[a]);
    if (accept_draw<CMP64>(acc[a], T[fsp - fs + 12])) {
      cnt = cnt + ohp - oh[a];
      oh[a] = ohp;
      m[a] = mp;
      t4[a] = tp;
      ++naccepted;
    }
  }
  if (count_pairs) {
#pragma unroll
    for (int a = 0; a < 4; ++a) pair_sum += nibble(cnt, m[a]);
  }
  cnt_out = cnt;
  uint32_t bonds = 0;
  if (BONDS) {
#pragma unroll
    for (int a = 0; a < 4; ++a) bonds += __umulhi(nb8[a] * m[a], 2u);
  }
  return bonds;
}

// 4*sigma of arm b of the 16-bit cell in half `hi` of a word.
__device__ __forceinline__ uint32_t arm4(uint32_t word, int hi, int b) {
  const int sh = 16 * hi + 3 * b - 2;
  return (sh >= 0) ? ((word >> sh) & 0x1Cu) : ((word << 2) & 0x1Cu);
}

// Philox key material of the lattice being swept: the precomputed round keys
// (single lattice) or the seed words, advanced in registers (batch, where
// consecutive tiles may belong to different replicas).
struct KeysRound {
  const RoundKeys* K;
};
struct KeysSeed {
  uint32_t k0, k1;
};

template <int RNG_WORDS>
__device__ __forceinline__ void draws(uint32_t c, uint32_t s_lo, uint32_t s_hi, const KeysRound& k,
                                      uint32_t q, uint32_t acc[4], uint32_t kk[4]) {
  cell_draws<RNG_WORDS>(c, s_lo, s_hi, *k.K, q, acc, kk);
}

template <int RNG_WORDS>
__device__ __forceinline__ void draws(uint32_t c, uint32_t s_lo, uint32_t s_hi, const KeysSeed& k,
                                      uint32_t q, uint32_t acc[4], uint32_t kk[4]) {
  const Words4 u = philox_seed(c, s_lo, s_hi, kTagAccept, k.k0, k.k1);
  const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
  if (RNG_WORDS == 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const uint64_t prod = (uint64_t)uw[a] * (uint64_t)(q - 1u);
      kk[a] = (uint32_t)(prod >> 32);
      acc[a] = (uint32_t)prod;
    }
  } else {
    const Words4 p = philox_seed(c, s_lo, s_hi, kTagPropose, k.k0, k.k1);
    const uint32_t pw[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      acc[a] = uw[a];
      kk[a] = __umulhi(pw[a], q - 1u);
    }
  }
}

// Update the cell in half `hi` of word `own`; xm / xp are the words to the
// left / right, ym / yp the words of the rows y-1 / y+1.
template <int RNG_WORDS, bool CMP64, bool BONDS, typename KEYS>
__device__ __forceinline__ uint32_t update_in_word(
    uint32_t own, uint32_t xm_word, uint32_t xp_word, uint32_t ym_word, uint32_t yp_word, int hi,
    uint32_t c, uint32_t s_lo, uint32_t s_hi, const KEYS& keys, uint32_t q,
    const ProposalTable& P, const typename ThresholdRow<CMP64>::type* T, uint32_t& nacc,
    uint32_t& pair_sum, uint32_t& bonds, uint32_t* s_hist4) {
  // partner arms: arm 0 (+x) <-> arm 1 of the +x cell, arm 1 (-x) <-> arm 0 of
  // the -x cell, arm 2 (+y) <-> arm 3 of the +y cell, arm 3 <-> arm 2 of -y
  uint32_t n4[4];
  if (hi) {
    n4[0] = arm4(xp_word, 0, 1);
    n4[1] = arm4(own, 0, 0);
  } else {
    n4[0] = arm4(own, 1, 1);
    n4[1] = arm4(xm_word, 1, 0);
  }
  n4[2] = arm4(yp_word, hi, 3);
  n4[3] = arm4(ym_word, hi, 2);
  uint32_t nb8[4], t4[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    nb8[a] = 8u << n4[a];
    t4[a] = arm4(own, hi, a);
  }
  uint32_t acc[4], kk[4];
  draws<RNG_WORDS>(c, s_lo, s_hi, keys, q, acc, kk);
  uint32_t cnt;
  // equal pairs (N_sigma) and N_q' only on recorded steps (s_hist4 set)
  bonds += update_arms_tab<CMP64, BONDS>(t4, nb8, acc, kk, P, T, nacc, pair_sum, cnt,
                                         s_hist4 != nullptr);
  if (s_hist4) hist_add_cell(s_hist4, cnt);
  const uint32_t wn = (t4[0] >> 2) | (t4[1] << 1) | (t4[2] << 4) | (t4[3] << 7);
  return hi ? ((own & 0xFFFFu) | (wn << 16)) : ((own & 0xFFFF0000u) | wn);
}

// Staged input: rows y0-2 .. y0+TR+1 and words p0-4 .. p0+TW+3 (a 16-byte
// aligned box, so one TMA copy can fill it); word p0-1+jj sits in column
// jj+3.  After colour 0: rows y0-1 .. y0+TR, words p0-1 .. p0+TW.
constexpr int kInColOff = 3;
template <int TR, int TW>
struct TileSmem {
  alignas(128) uint32_t in[TR + 4][TW + 8];
  uint32_t mid[TR + 2][TW + 2];
};

// Per-thread counts of the cells a thread finished inside its tiles:
// pair_sum adds 4 + 2 (equal pairs) per counted cell.
struct TileCounts {
  uint32_t pair_sum, ncells, bonds, nacc;
  __device__ __forceinline__ uint32_t pairs() const { return (pair_sum - 4u * ncells) >> 1; }
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
      S.in[rr][jj + kInColOff] = CG ? __ldcg(row + p) : row[p];
    }
  }
}

// Colour 0: tile rows -1 .. th, words 0 .. tw-1 (the colour-0 cell of a word
// is its low half on even rows, its high half on odd rows), then the one
// colour-0 cell per row just outside the tile (x0 - 1, high half of word -1,
// on odd rows; x0 + 2 tw, low half of word tw, on even rows).  Reads S.in,
// writes S.mid.  s_hist4 != nullptr (recorded steps): N_q' and the equal
// pairs of the tile's cells are counted.
template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, typename KEYS>
__device__ __forceinline__ void colour0(const StepView<KEYS>& v, const TileGeom& g,
                                        TileSmem<TR, TW>& S, const ProposalTable& P,
                                        const typename ThresholdRow<CMP64>::type* T,
                                        TileCounts& cnt, uint32_t* s_hist4) {
  constexpr int kRows = (TW >= 32) ? 1 : 32 / TW;  // rows per warp pass
  constexpr int kLanes = (TW >= 32) ? 32 : TW;     // lanes per row
  constexpr int C = kInColOff + 1;                 // column of word 0
  const int L = v.L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lrow = lane / kLanes, lcol = lane % kLanes;
  const int th = g.th, tw = g.tw, y0 = g.y0, p0 = g.p0;
  for (int r0 = warp * kRows - 1; r0 <= th; r0 += (NT / 32) * kRows) {
    const int r = r0 + lrow;
    if (r > th) continue;
    const int y = y0 + r;
    const int hi = y & 1;
    const int yg = (y < 0) ? y + L : (y >= L ? y - L : y);
    const bool inside = (r >= 0) && (r < th);
    for (int j = lcol; j < tw; j += kLanes) {
      const int xg = 2 * (p0 + j) + hi;
      uint32_t dummy = 0, dummy_b = 0;
      const uint32_t out = update_in_word<RNG_WORDS, CMP64, false>(
          S.in[r + 2][j + C], S.in[r + 2][j + C - 1], S.in[r + 2][j + C + 1],
          S.in[r + 1][j + C], S.in[r + 3][j + C], hi, (uint32_t)((long long)yg * L + xg),
          v.s_lo, v.s_hi, v.keys, v.q, P, T, inside ? cnt.nacc : dummy,
          inside ? cnt.pair_sum : dummy, dummy_b, inside ? s_hist4 : nullptr);
      if (inside) ++cnt.ncells;
      S.mid[r + 1][j + 1] = out;
    }
  }
  // the ring goes to the warps after the first two, which take one row of
  // the th + 2 fewer than warps 0 and 1 when 8 warps share 66 rows
  const int ring0 = (NT >= 128 && TW >= 32) ? 64 : 0;
  for (int i = (int)threadIdx.x - ring0; i < th + 2; i += NT) {
    if (i < 0) continue;
    const int r = i - 1;
    const int y = y0 + r;
    const int hi = y & 1;
    const int j = hi ? -1 : tw;
    const int yg = (y < 0) ? y + L : (y >= L ? y - L : y);
    int xg = 2 * (p0 + j) + hi;
    xg = (xg < 0) ? xg + L : (xg >= L ? xg - L : xg);
    uint32_t d0 = 0, d1 = 0, d2 = 0;
    // the unused side of the ring word is clamped into the staged columns
    const int jm = max(j, 0), jp = min(j + 2, tw + 1);
    S.mid[r + 1][j + 1] = update_in_word<RNG_WORDS, CMP64, false>(
        S.in[r + 2][j + C], S.in[r + 2][jm + kInColOff], S.in[r + 2][jp + kInColOff],
        S.in[r + 1][j + C], S.in[r + 3][j + C], hi, (uint32_t)((long long)yg * L + xg), v.s_lo,
        v.s_hi, v.keys, v.q, P, T, d0, d1, d2, nullptr);
  }
}

// Colour 1: tile rows 0 .. th-1 (low half on odd rows, high on even rows),
// from S.mid to the destination buffer.
template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, typename KEYS>
__device__ __forceinline__ void colour1(const StepView<KEYS>& v, const TileGeom& g,
                                        TileSmem<TR, TW>& S, const ProposalTable& P,
                                        const typename ThresholdRow<CMP64>::type* T,
                                        TileCounts& cnt, uint32_t* s_hist4) {
  constexpr int kRows = (TW >= 32) ? 1 : 32 / TW;
  constexpr int kLanes = (TW >= 32) ? 32 : TW;
  const int L = v.L, Lh = v.Lh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lrow = lane / kLanes, lcol = lane % kLanes;
  const int th = g.th, tw = g.tw, y0 = g.y0, p0 = g.p0;
  for (int r0 = warp * kRows; r0 < th; r0 += (NT / 32) * kRows) {
    const int r = r0 + lrow;
    if (r >= th) continue;
    const int y = y0 + r;
    const int hi = (y & 1) ^ 1;
    uint32_t* drow = v.dst + (size_t)y * Lh + p0;
    for (int j = lcol; j < tw; j += kLanes) {
      const int xg = 2 * (p0 + j) + hi;
      drow[j] = update_in_word<RNG_WORDS, CMP64, true>(
          S.mid[r + 1][j + 1], S.mid[r + 1][j], S.mid[r + 1][j + 2], S.mid[r][j + 1],
          S.mid[r + 2][j + 1], hi, (uint32_t)((long long)y * L + xg), v.s_lo, v.s_hi, v.keys,
          v.q, P, T, cnt.nacc, cnt.pair_sum, cnt.bonds, s_hist4);
      ++cnt.ncells;
    }
  }
}

// Sweep the tile at rows y0.., words p0.. of one lattice with synchronous
// staging.  Called by all threads of the block; ends with the tile written
// to dst (no trailing barrier: the caller synchronises before reusing the
// shared buffers).  s_hist4 != nullptr (recorded steps): N_q' of the tile's
// cells is added to hist_out[0..8) through the block's four zeroed shared
// words, and the equal pairs (N_sigma) are counted; on other steps neither
// is (N_HB_raw, which the volume move needs, and the accepted moves are
// counted on every step).  A warp covers max(1, 32/TW) rows per pass.
template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT, typename KEYS, bool CG = false>
__device__ __forceinline__ void sweep_tile(const StepView<KEYS>& v, int y0, int p0,
                                           TileSmem<TR, TW>& S, const ProposalTable& P,
                                           const typename ThresholdRow<CMP64>::type* T,
                                           TileCounts& cnt, uint32_t* s_hist4,
                                           unsigned long long* hist_out) {
  static_assert(TW >= 32 ? (TW % 32 == 0) : (32 % TW == 0), "tile width");
  const TileGeom g = tile_geom<TR, TW>(v.L, v.Lh, y0, p0);
  stage_plain<TR, TW, NT, CG>(v, g, S);
  __syncthreads();
  colour0<RNG_WORDS, CMP64, TR, TW, NT>(v, g, S, P, T, cnt, s_hist4);
  __syncthreads();
  colour1<RNG_WORDS, CMP64, TR, TW, NT>(v, g, S, P, T, cnt, s_hist4);
  if (s_hist4) {  // block-uniform: only on recorded steps
    __syncthreads();
    hist_flush(s_hist4, hist_out);
  }
}

}  // namespace cvf
