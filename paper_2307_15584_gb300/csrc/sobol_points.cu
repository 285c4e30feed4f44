// sobol_points.cu -- materialised Sobol' points (HBM-write bound): Alg. 3 /
// Eq. (ts), y_j(i) = XOR of the generator columns selected by the bits of i,
// randomised in integers (Sec. 2.3), mapped to [0,1) (Sec. 2.1); 32-bit, 64-bit
// (Alg. 3's wide indices) and partitioned (Sec. 2.5.1) enumeration.
//
// Fast path layout.  Output rows are [count][s] u32/f32.  A warp writes a
// "group" of Q = 128 / gcd(s,128) consecutive points per step: Q*s = 128*K
// elements, i.e. K 16-byte chunks per lane, so every store is a coalesced
// 128-bit store.  Lane l owns chunks l, l+32, .. of the group; element e of
// a group is point p_e = e / s, dimension j_e = e % s, the same in every group.
//
// Linearity over GF(2) makes the per-element cost O(1): for a group starting
// at enumeration index G*Q (index_begin is a multiple of Q: a range that starts
// off that grid sends its first rows, up to the next multiple of Q, through the
// one-element-per-thread kernel), the bits of the enumeration index J split into three
// disjoint fields,
//   J = (G_hi << (u + q)) | (G_in << q) | p_e,   G_in < 2^u, p_e < Q,
// and y_j(i) = Hout_j(G_hi) ^ Hin_j[G_in] ^ lo_e for i = (J << col0) | pconst.
// lo_e (which also carries the fixed low part pconst) is fixed per lane, Hin
// is a shared-memory table of 2^u rows, and Hout changes once every 2^u groups,
// by the columns of the G_hi bits that flip.  G_hi takes up to 64 bits (Alg. 3's
// wide indices).
#include <cstdint>

#include "points_common.cuh"

namespace qmc {

namespace {
using namespace pts;

// Fills tab[r][j] (row stride s) for r < rows, a power of two: the XOR of the columns c0 + b of
// dimension j over the set bits b of r (columns at or above m count as zero), by doubling --
// rows [2^b, 2^(b+1)) are rows [0, 2^b) with column c0 + b added.  cols: [s][ms] in shared
// memory.  Ends with a block barrier.
__device__ void fill_index_table(uint32_t* tab, uint32_t rows, uint32_t s, const uint32_t* cols, uint32_t ms,
                                 uint32_t m, uint32_t c0) {
  const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31u;
  for (uint32_t j = threadIdx.x; j < s; j += blockDim.x) tab[j] = 0u;
  __syncthreads();
  for (uint32_t half = 1, b = 0; half < rows; half <<= 1, ++b) {
    for (uint32_t r = warp; r < half; r += nwarps)
      for (uint32_t j = lane; j < s; j += 32u)
        tab[(half + r) * s + j] = tab[r * s + j] ^ (c0 + b < m ? cols[j * ms + c0 + b] : 0u);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K1 fast path.  MODE: 0 none, 1 XOR, 2 nested (a.scramble = NESTED_XOR adds the
// digital shift before the nested scramble, folded into the fixed per-lane terms).
// K: 16-byte chunks per lane.
// Shared memory: cols[s][m + 1] (mirrored for nested; rows padded by one word so
// that lanes reading one column of consecutive dimensions hit distinct banks),
// hin[2^u][s], pc[s].  Table entries for index bits at or above m stay zero: no
// enumerated index sets them.
// ---------------------------------------------------------------------------
// TMA: full groups go through a WarpStager (bulk stores from shared memory).
template <int K, int MODE, bool V4, bool TMA>  // V4: s % 4 == 0, chunks hold 4 consecutive dimensions
__global__ void __launch_bounds__(kThreads) sobol_points_fast(PointsArgs a) {
  extern __shared__ __align__(128) uint32_t smem[];
  const uint32_t s = a.s;
  const uint32_t nin = 1u << a.u_log2;
  // [warps][WarpStager words], then the tables
  uint32_t* cols = smem + (TMA ? (kThreads / 32) * WarpStager<K>::kWarpWords : 0);
  const uint32_t m = a.m, ms = m + 1u;
  uint32_t* hin = cols + s * ms;
  uint32_t* pc = hin + nin * s;

  for (uint32_t idx = threadIdx.x; idx < s * m; idx += blockDim.x) {
    const uint32_t c = __ldg(a.matrices + idx), j = idx / m;
    cols[idx + j] = (MODE == 2) ? __brev(c) : c;
  }
  __syncthreads();
  const uint32_t cin = a.col0 + a.q_log2;  // column of the lowest G_in bit
  fill_index_table(hin, nin, s, cols, ms, m, cin);
  for (uint32_t j = threadIdx.x; j < s; j += blockDim.x) {
    uint32_t y = 0;
    for (uint32_t k = 0; k < a.col0; ++k)
      if ((a.pconst >> k) & 1u) y ^= cols[j * ms + k];
    pc[j] = y;
  }
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t Q = 1u << a.q_log2;
  uint32_t jd[4 * K], lo[4 * K], hout[4 * K];
  NestedKey key[4 * K];
#pragma unroll
  for (int c = 0; c < K; ++c)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t e = 4u * (lane + 32u * c) + t;
      const uint32_t p = e / s, j = e - p * s;
      uint32_t y = pc[j];
      for (uint32_t k = 0; k < a.q_log2 && a.col0 + k < m; ++k)
        if ((p >> k) & 1u) y ^= cols[j * ms + a.col0 + k];
      if (MODE == 1) y ^= __ldg(a.seeds + j);
      if (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR) y ^= __brev(__ldg(a.seeds + j));  // mirrored shift
      jd[4 * c + t] = j;
      lo[4 * c + t] = y;
      key[4 * c + t] = nested_key(MODE == 2 ? __ldg(a.seeds + j) : 0u);
    }

  const uint64_t n_groups = (a.count + Q - 1) >> a.q_log2;
  const uint64_t full_groups = a.count >> a.q_log2;  // groups whose Q rows all exist
  uint64_t g0, g1;
  warp_range(n_groups, g0, g1);
  const uint64_t G_first = a.index_begin >> a.q_log2;
  const uint32_t hi_col = a.col0 + a.q_log2 + a.u_log2;  // column of the lowest G_hi bit
  const uint64_t step = (uint64_t)Q * s;  // elements per group
  uint64_t off = g0 * step + 4u * lane;   // this lane's first element in group g0

  WarpStager<K> stager(smem + (threadIdx.x >> 5) * WarpStager<K>::kWarpWords);

  for (uint64_t g = g0; g < g1; ++g, off += step) {
    const uint64_t G = G_first + g;
    const uint32_t G_in = (uint32_t)G & (nin - 1u);
    if (g == g0) {
      const uint64_t G_hi = G >> a.u_log2;  // below 2^(m - hi_col) for every enumerated group
#pragma unroll
      for (int e = 0; e < 4 * K; ++e) {
        uint32_t y = 0;
        for (uint32_t k = 0; (G_hi >> k) != 0; ++k)
          if ((G_hi >> k) & 1u) y ^= cols[jd[e] * ms + hi_col + k];
        hout[e] = y;
      }
    } else if (G_in == 0) {
      // G_hi advanced by one: exactly the bits of G_hi ^ (G_hi - 1) flipped
      // (the trailing ones and the bit above them), two on average.
      const uint64_t G_hi = G >> a.u_log2;
      const uint32_t nflip = (uint32_t)__ffsll((long long)G_hi);  // G_hi > 0 here
#pragma unroll
      for (int e = 0; e < 4 * K; ++e) {
        uint32_t y = hout[e];
        for (uint32_t k = 0; k < nflip; ++k) y ^= cols[jd[e] * ms + hi_col + k];
        hout[e] = y;
      }
    }
    const uint32_t* hrow = hin + G_in * s;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      uint32_t h[4];
      if (V4) {  // four consecutive dimensions: one 128-bit shared-memory load
        const uint4 q = *reinterpret_cast<const uint4*>(hrow + jd[4 * c]);
        h[0] = q.x, h[1] = q.y, h[2] = q.z, h[3] = q.w;
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) h[t] = hrow[jd[4 * c + t]];
      }
      uint32_t v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        uint32_t y = h[t] ^ hout[4 * c + t] ^ lo[4 * c + t];
        if (MODE == 2) y = __brev(nested_mix(y, key[4 * c + t]));
        v[t] = y;
      }
      const uint64_t o = off + 128u * c;
      if (g < full_groups) {
        if (TMA)
          stager.put(lane, c, v);
        else
          store4(a.out_u32, a.out_f32, o, v, a.chk);
      } else {  // ragged last group: per-element row test
        const uint64_t rows_left = a.count - (g << a.q_log2);
        const uint32_t e0 = 4u * (lane + 32u * c);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if ((uint64_t)((e0 + t) / s) < rows_left) store1(a.out_u32, a.out_f32, o + t, v[t], a.chk);
      }
    }
    if (TMA && g < full_groups)
      stager.group_done(lane, off, g + 1 == g1 || g + 1 == full_groups, a.out_u32, a.out_f32);
  }
  if (TMA) stager.finish(lane);
}

// K1 walking path, for what the fast path's 16-byte groups do not fit (s / gcd(s, 128) > 4,
// index_begin * s not a multiple of 4, outputs off a 16-byte boundary).  A warp takes a chunk of
// consecutive output dimensions (w of them) and walks it down the rows: with the
// enumeration index J = (J_hi << u) | J_lo, y_j = pc_j ^ Hlo_j[J_lo] ^ Hhi_j(J_hi), Hlo a
// shared-memory table of 2^u rows (u >= 5) and Hhi changed, when J_lo wraps, by the columns of
// the J_hi bits that flip.
//
// With 16-byte aligned rows (s % 4 == 0 and aligned outputs) chunks are up to 128 dimensions
// wide and lanes own quads of four dimensions: with nq = w / 4 quads per row of the chunk, lane l
// holds dimensions 4 (l % nq) .. + 3 of rows l / nq, + kq, .. (kq = floor(32 / nq) rows per warp
// step), so a warp step writes kq consecutive rows of an s <= 128 output as one contiguous span;
// each lane reads the four table entries of a row with one 16-byte shared-memory load and writes
// them with one 16-byte store per output; two steps go together (2 kq <= 2^u: they wrap J_lo at
// most once), their loads in flight at once.
// Otherwise lanes own dimensions, lane l holding dimension l mod w of rows l / w, + k, ..
// (k = floor(32 / w)), in groups of four steps with 4-byte stores: the four table reads of a
// group do not depend on one another or on Hhi, so they are in flight together, and the group's
// rows past a wrap take the advanced Hhi (4 k <= 2^u; a 32-wide chunk, k = 1, reads rows
// J_lo .. J_lo + 3 of a table that repeats its first three rows after the last, so its reads
// need no wrap).
constexpr uint32_t kWalkSteps = 256;
constexpr uint32_t kWalkExtraRows = 3;  // copies of table rows 0-2 after the last row

template <int MODE>
__global__ void __launch_bounds__(kThreads) sobol_points_walk(PointsArgs a) {
  extern __shared__ __align__(128) uint32_t smem[];
  const uint32_t s = a.s, m = a.m, ms = m + 1u, u = a.u_log2, nlo = 1u << u;
  uint32_t* cols = smem;                        // [s][m + 1], mirrored for nested, padded rows
  uint32_t* hlo = cols + s * ms;                // [2^u + 3][s]
  uint32_t* pc = hlo + (nlo + kWalkExtraRows) * s;  // [s]: the fixed low index part
  for (uint32_t idx = threadIdx.x; idx < s * m; idx += blockDim.x) {
    const uint32_t c = __ldg(a.matrices + idx), j = idx / m;
    cols[idx + j] = (MODE == 2) ? __brev(c) : c;  // row j starts at j (m + 1)
  }
  __syncthreads();
  fill_index_table(hlo, nlo, s, cols, ms, m, a.col0);
  for (uint32_t idx = threadIdx.x; idx < kWalkExtraRows * s; idx += blockDim.x) hlo[nlo * s + idx] = hlo[idx];
  for (uint32_t j = threadIdx.x; j < s; j += blockDim.x) {
    uint32_t y = 0;
    for (uint32_t b = 0; b < a.col0; ++b)
      if ((a.pconst >> b) & 1u) y ^= cols[j * ms + b];
    pc[j] = y;
  }
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31u;
  const bool rows16 = (s & 3u) == 0 && (((uintptr_t)a.out_u32 | (uintptr_t)a.out_f32) & 15u) == 0;
  // chunks of cw dimensions, 32 lanes per row of a whole chunk: 32 quads (128 dimensions) with
  // 16-byte rows, else 32 dimensions; the last chunk is wl wide, kl rows per warp step
  const uint32_t cw = rows16 ? 128u : 32u;
  const uint32_t nch = (s + cw - 1u) / cw, wl = s - cw * (nch - 1u), kl = 32u / (rows16 ? wl >> 2 : wl);
  // Units go by row blocks of Ul rows: kl units of kWalkSteps rows per full chunk, then one unit of
  // the last chunk, so the chunks of the same rows -- which share cache lines where a row is not a
  // whole number of lines -- are written at about the same time.
  const uint64_t Ul = (uint64_t)kWalkSteps * kl;
  const uint32_t per_block = (nch - 1u) * kl + 1u;
  const uint64_t n_units = (a.count + Ul - 1) / Ul * per_block;
  const uint32_t hi_col = a.col0 + u;  // column of the lowest J_hi bit
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t un = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); un < n_units; un += nw) {
    const uint64_t rb = un / per_block;
    const uint32_t within = (uint32_t)(un - rb * per_block);
    const bool last = within == per_block - 1u;
    const uint32_t c = last ? nch - 1u : within / kl;
    const uint32_t w = last ? wl : cw, k = last ? kl : 1u;
    const uint64_t U = last ? Ul : (uint64_t)kWalkSteps;
    const uint64_t r0 = rb * Ul + (last ? 0u : (uint64_t)(within - c * kl) * kWalkSteps);
    if (r0 >= a.count) continue;  // the last row block is cut by the range
    if (rows16) {
      // nq = w / 4 quads of dimensions per row, kq = k = floor(32 / nq) rows per step: lane l takes
      // dimensions jq .. jq + 3 (jq = 128 c + 4 (l % nq)) of rows r0 + l / nq, + kq, ..
      const uint32_t nq = w >> 2, kq = k;
      if (lane >= nq * kq) continue;  // nq does not divide 32: the remaining lanes idle
      const uint32_t jq = cw * c + 4u * (lane % nq), qr = lane / nq;
      const uint64_t r_end = r0 + U < a.count ? r0 + U : a.count;
      if (r0 + qr >= r_end) continue;
      const uint32_t steps = ((uint32_t)(r_end - r0 - qr) + kq - 1u) / kq;
      const uint64_t J = a.index_begin + r0 + qr;
      uint32_t jlo = (uint32_t)J & (nlo - 1u);
      uint64_t jhi = J >> u;
      uint32_t base[4];
      NestedKey key[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t* cj = cols + (jq + i) * ms;
        uint32_t h = pc[jq + i];
        for (uint32_t b = 0; (jhi >> b) != 0 && hi_col + b < m; ++b)
          if ((jhi >> b) & 1u) h ^= cj[hi_col + b];
        const uint32_t seed = MODE != 0 ? __ldg(a.seeds + jq + i) : 0u;
        if (MODE == 1) h ^= seed;
        if (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR) h ^= __brev(seed);  // the shift, mirrored
        base[i] = h;
        key[i] = nested_key(seed);
      }
      const uint32_t* hq = hlo + jq;
      const uint32_t dq = kq * s;       // elements per step
      uint64_t o = (r0 + qr) * s + jq;  // this lane's chunk of the current row
      auto emit = [&](const uint4 hv, const uint32_t (&b)[4]) {
        uint32_t v[4] = {hv.x ^ b[0], hv.y ^ b[1], hv.z ^ b[2], hv.w ^ b[3]};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (MODE == 2) v[i] = __brev(nested_mix(v[i], key[i]));
        store4(a.out_u32, a.out_f32, o, v, a.chk);
        o += dq;
      };
      auto advance4 = [&](uint32_t (&b)[4]) {  // J_hi advances by one: the bits of jhi ^ (jhi + 1) flip
        ++jhi;
        const uint32_t nflip = (uint32_t)__ffsll((long long)jhi);  // jhi > 0
        for (uint32_t bb = 0; bb < nflip && hi_col + bb < m; ++bb)
#pragma unroll
          for (int i = 0; i < 4; ++i) b[i] ^= cols[(jq + i) * ms + hi_col + bb];
      };
      uint32_t t = 0;
      if (2u * kq <= nlo) {  // two steps at once: J_lo + kq and J_lo + 2 kq wrap at most once
        for (; t + 2u <= steps; t += 2u) {
          const uint4 h0 = *reinterpret_cast<const uint4*>(hq + jlo * s);
          const uint4 h1 = *reinterpret_cast<const uint4*>(hq + ((jlo + kq) & (nlo - 1u)) * s);
          uint32_t nb[4] = {base[0], base[1], base[2], base[3]};
          if (jlo + 2u * kq >= nlo) advance4(nb);  // in or right after these two steps
          emit(h0, base);
          const bool second_past = jlo + kq >= nlo;
          uint32_t b1[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) b1[i] = second_past ? nb[i] : base[i];
          emit(h1, b1);
#pragma unroll
          for (int i = 0; i < 4; ++i) base[i] = nb[i];
          jlo = (jlo + 2u * kq) & (nlo - 1u);
        }
      }
      for (; t < steps; ++t) {  // kq <= 32 <= 2^u: one step wraps J_lo at most once
        emit(*reinterpret_cast<const uint4*>(hq + jlo * s), base);
        jlo += kq;
        if (jlo >= nlo) {
          jlo -= nlo;
          advance4(base);
        }
      }
      continue;
    }
    if (lane >= k * w) continue;  // w does not divide 32: the remaining lanes idle
    const uint32_t jo = 32u * c + lane % w;
    const uint64_t row = r0 + lane / w;
    const uint64_t r_end = r0 + U < a.count ? r0 + U : a.count;
    if (row >= r_end) continue;
    const uint32_t steps = ((uint32_t)(r_end - row) + k - 1) / k;  // r_end - row <= U <= kWalkSteps k
    const uint64_t J = a.index_begin + row;
    uint32_t jlo = (uint32_t)J & (nlo - 1u);
    uint64_t jhi = J >> u;
    const uint32_t* cj = cols + jo * ms;
    uint32_t base = pc[jo];
    for (uint32_t b = 0; (jhi >> b) != 0 && hi_col + b < m; ++b)
      if ((jhi >> b) & 1u) base ^= cj[hi_col + b];
    const uint32_t seed = MODE != 0 ? __ldg(a.seeds + jo) : 0u;
    if (MODE == 1) base ^= seed;
    if (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR) base ^= __brev(seed);  // the shift, mirrored
    const NestedKey key = nested_key(seed);
    // the unit's outputs from its first row on: at most kWalkSteps k s <= 2^23 elements (s <= 1024)
    const uint64_t off0 = row * s + jo;
    const uint32_t dofs = k * s;
    uint32_t ofs = 0, t = 0;
    // Hhi after J_hi advances by one: the bits of jhi ^ (jhi + 1) flip
    auto advance = [&](uint32_t h) {
      ++jhi;
      const uint32_t nflip = (uint32_t)__ffsll((long long)jhi);  // jhi > 0
      for (uint32_t b = 0; b < nflip && hi_col + b < m; ++b) h ^= cj[hi_col + b];
      return h;
    };
    auto finish = [&](uint32_t y) { return MODE == 2 ? __brev(nested_mix(y, key)) : y; };
    auto store_rows = [&](const uint32_t (&y4)[4]) {  // 4-byte stores of four steps
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t o = ofs + (uint32_t)q * dofs;
        if (in_bounds(a.chk, off0 + o, 1, kCheckPoints)) {
          if (a.out_u32) a.out_u32[off0 + o] = y4[q];
          if (a.out_f32) a.out_f32[off0 + o] = map_u32_to_unifloat(y4[q]);
        }
      }
    };
    if (w == 32u) {  // k = 1
      const uint32_t* hp = hlo + jo;
      const uint32_t s2 = 2u * s, s3 = 3u * s;
      for (; t + 4u <= steps; t += 4u) {
        const uint32_t* hr = hp + jlo * s;
        uint32_t y4[4] = {hr[0], hr[s], hr[s2], hr[s3]};
        const uint32_t left = nlo - jlo;  // steps before J_hi advances, >= 1
        const uint32_t next = left <= 4u ? advance(base) : base;
#pragma unroll
        for (int q = 0; q < 4; ++q) y4[q] = finish(y4[q] ^ ((uint32_t)q < left ? base : next));
        base = next;
        jlo = (jlo + 4u) & (nlo - 1u);
        store_rows(y4);
        ofs += 4u * s;
      }
    } else if (4u * k <= nlo) {
      for (; t + 4u <= steps; t += 4u) {
        uint32_t y4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) y4[q] = hlo[((jlo + (uint32_t)q * k) & (nlo - 1u)) * s + jo];
        const bool adv = jlo + 4u * k >= nlo;
        const uint32_t next = adv ? advance(base) : base;
#pragma unroll
        for (int q = 0; q < 4; ++q) y4[q] = finish(y4[q] ^ (jlo + (uint32_t)q * k >= nlo ? next : base));
        base = next;
        jlo = (jlo + 4u * k) & (nlo - 1u);
        store_rows(y4);
        ofs += 4u * dofs;
      }
    }
    for (; t < steps; ++t) {  // the unit's last steps, one at a time
      const uint32_t y = finish(hlo[jlo * s + jo] ^ base);
      if (in_bounds(a.chk, off0 + ofs, 1, kCheckPoints)) {
        if (a.out_u32) a.out_u32[off0 + ofs] = y;
        if (a.out_f32) a.out_f32[off0 + ofs] = map_u32_to_unifloat(y);
      }
      ofs += dofs;
      jlo += k;
      if (jlo >= nlo) {
        jlo -= nlo;
        base = advance(base);
      }
    }
  }
}

// K1 generic path: one element per thread, columns read through the cache.
template <int MODE>
__global__ void __launch_bounds__(kThreads) sobol_points_generic(PointsArgs a) {
  const uint64_t total = a.count * a.s;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += stride) {
    const uint64_t r = f / a.s;
    const uint32_t j = (uint32_t)(f - r * a.s);
    uint64_t i = ((a.index_begin + r) << a.col0) | a.pconst;  // below 2^m (checked by the caller)
    const uint32_t* Cj = a.matrices + (uint64_t)j * a.m;
    uint32_t y = 0;
    for (; i != 0; i &= i - 1u) y ^= __ldg(Cj + (__ffsll((long long)i) - 1));
    if (MODE == 1 || (MODE == 2 && a.scramble == QMC_SCRAMBLE_NESTED_XOR)) y ^= __ldg(a.seeds + j);
    if (MODE == 2) y = __brev(nested_mix(__brev(y), nested_key(__ldg(a.seeds + j))));
    store1(a.out_u32, a.out_f32, f, y, a.chk);
  }
}

}  // namespace

// One element per thread, the columns read through the cache.
static cudaError_t launch_sobol_generic(const PointsArgs& a, cudaStream_t stream) {
  switch (a.scramble) {
    case 0: return launch_grid_stride(sobol_points_generic<0>, a.count * a.s, stream, a);
    case 1: return launch_grid_stride(sobol_points_generic<1>, a.count * a.s, stream, a);
    default: return launch_grid_stride(sobol_points_generic<2>, a.count * a.s, stream, a);
  }
}

// The walking kernel, or the generic one for tables beyond shared memory.
static cudaError_t launch_sobol_walk(PointsArgs a, cudaStream_t stream) {
  const size_t optin = device_info().smem_per_block_optin;
  // the columns (rows padded by one word), a low table of 2^w + 3 rows (5 <= w <= 8) and pc
  auto walk_words = [&](uint32_t w) {
    return (size_t)a.s * (a.m + 1) + (((size_t)1 << w) + kWalkExtraRows) * a.s + a.s;
  };
  uint32_t w = 8;
  while (w > 5 && walk_words(w) * sizeof(uint32_t) > optin) --w;
  const size_t walk_smem = walk_words(w) * sizeof(uint32_t);
  if (walk_smem <= optin && a.s <= 1024) {
    a.u_log2 = w;
    // the kernel's chunk geometry: 128-dimension chunks of quads with 16-byte rows, else 32
    const bool rows16 = (a.s & 3u) == 0 && aligned16(a.out_u32) && aligned16(a.out_f32);
    const uint32_t cw = rows16 ? 128u : 32u;
    const uint32_t nch = (a.s + cw - 1u) / cw, wl = a.s - cw * (nch - 1u), kl = 32u / (rows16 ? wl >> 2 : wl);
    const uint64_t Ul = (uint64_t)kWalkSteps * kl;
    const uint64_t units = (a.count + Ul - 1) / Ul * ((nch - 1u) * kl + 1u);
    // one unit per warp on a grid sized by the units (launch_spread): at s = 40 this wrote 9 %
    // faster than a persistent grid striding over the units; the table build per block is a few
    // percent of a block's work
    switch (a.scramble) {
      case 0: return launch_spread(sobol_points_walk<0>, units, 1, walk_smem, stream, a);
      case 1: return launch_spread(sobol_points_walk<1>, units, 1, walk_smem, stream, a);
      default: return launch_spread(sobol_points_walk<2>, units, 1, walk_smem, stream, a);
    }
  }
  return launch_sobol_generic(a, stream);
}

cudaError_t launch_sobol_points(PointsArgs a, cudaStream_t stream) {
  const uint32_t K = fast_k(a.s);
  a.q_log2 = log2_exact(K ? 128u * K / a.s : 1u);
  // index_begin * s a multiple of 4: the group grid's rows start on 16-byte boundaries of the output
  bool fast = K != 0 && a.s <= 256 && ((a.index_begin * a.s) & 3u) == 0 && aligned16(a.out_u32) &&
              aligned16(a.out_f32);
  // inner table of at most 16 KiB and 256 rows
  uint32_t u = 0;
  while (u < 8 && (2u << u) * a.s * 4u <= 16384u) ++u;
  a.u_log2 = u;
  // TMA bulk stores target device memory; outputs in host memory that the GPU
  // writes directly (pinned, mapped) take the 128-bit store path.
  bool tma = kPointsTma && device_resident(a.out_u32) && device_resident(a.out_f32);
  const size_t table_words = (size_t)a.s * (a.m + 1) + ((size_t)1 << u) * a.s + a.s;
  const size_t stage_words = (size_t)(kThreads / 32) * 4 * kStageGroups * 128u * K;
  const size_t optin = device_info().smem_per_block_optin;
  if (tma && (stage_words + table_words) * sizeof(uint32_t) > optin) tma = false;
  if (table_words * sizeof(uint32_t) > optin) fast = false;
  if (!fast) return launch_sobol_walk(a, stream);
  // a start off the group grid: the rows up to its next multiple of Q (fewer than 128) take the
  // one-element-per-thread kernel, the rest the fast path from there (an output offset of
  // head * s elements, 16-byte aligned)
  const uint64_t Q = 1ull << a.q_log2;
  const uint64_t head = (Q - (a.index_begin & (Q - 1u))) & (Q - 1u);
  if (head) {
    PointsArgs h = a;
    h.count = head < a.count ? head : a.count;
    const cudaError_t e = launch_sobol_generic(h, stream);
    if (e != cudaSuccess || h.count == a.count) return e;
    const uint64_t skip = h.count * a.s;
    a.index_begin += h.count;
    a.count -= h.count;
    if (a.out_u32) a.out_u32 += skip;
    if (a.out_f32) a.out_f32 += skip;
    a.chk.limit = a.chk.limit > skip ? a.chk.limit - skip : 0;
  }
  const size_t smem = ((tma ? stage_words : 0) + table_words) * sizeof(uint32_t);
  const uint64_t groups = (a.count + (1u << a.q_log2) - 1) >> a.q_log2;
  const bool v4 = (a.s & 3u) == 0;
  // direct stores: short per-warp ranges (launch_spread), long enough to pay each warp's first
  // Hout (one column XOR per set bit of G_hi) and each block's tables; 64 groups for the
  // sequences of up to 2^16 G_hi values, 256 for longer indices (measured at s = 32: 64-bit
  // indices at 2^40 ran 4 % slower with 64 groups a warp than with 256)
  uint32_t hb = 0;  // bit length of the largest G_hi
  for (uint64_t gh = ((a.index_begin + a.count) >> a.q_log2) >> a.u_log2; gh; gh >>= 1) ++hb;
  const uint64_t per_warp = hb <= 16 ? 64 : 256;
#define QMC_SOBOL_LAUNCH(T, KERNEL)                                 \
  ((T) ? launch_persistent(KERNEL, groups, smem, stream, a)         \
       : launch_spread(KERNEL, groups, per_warp, smem, stream, a))
#define QMC_SOBOL_MODES(KK, V, T)                                                 \
  if (a.scramble == 0) return QMC_SOBOL_LAUNCH(T, (sobol_points_fast<KK, 0, V, T>)); \
  if (a.scramble == 1) return QMC_SOBOL_LAUNCH(T, (sobol_points_fast<KK, 1, V, T>)); \
  return QMC_SOBOL_LAUNCH(T, (sobol_points_fast<KK, 2, V, T>));
#define QMC_SOBOL_CASE(KK)                \
  case KK:                                \
    if (v4 && tma) {                      \
      QMC_SOBOL_MODES(KK, true, kPointsTma)  \
    } else if (v4) {                      \
      QMC_SOBOL_MODES(KK, true, false)    \
    } else if (tma) {                     \
      QMC_SOBOL_MODES(KK, false, kPointsTma) \
    } else {                              \
      QMC_SOBOL_MODES(KK, false, false)   \
    }
  switch (K) {
    QMC_SOBOL_CASE(1)
    QMC_SOBOL_CASE(2)
    QMC_SOBOL_CASE(3)
    QMC_SOBOL_CASE(4)
    default: return cudaErrorInvalidValue;
  }
#undef QMC_SOBOL_CASE
#undef QMC_SOBOL_MODES
#undef QMC_SOBOL_LAUNCH
}

}  // namespace qmc
