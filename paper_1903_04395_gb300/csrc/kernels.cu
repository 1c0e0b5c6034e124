// kernels.cu - device side of one color-coding iteration (Section 2.1) in the
// linear-algebra form of Section 4: per DP step an SpMM P = A * M_p (Eq. 2,
// pre-computed neighbour traversal of Section 4.2, SpMM of Section 4.5) and
// an element-wise multiply-add over the color-set splits (eMA, Section 4.5),
// and at the last step a reduction over vertices.
//
// Relative-color tables.  N(v, T_s, C) is zero unless C contains c(v) (the
// root of T_s sits on v), and P(v, C_p) is only ever read for C_p without
// c(v) (C_p and the active child's set are disjoint and the latter holds
// c(v)).  So every row of vertex v is indexed by subsets of the K = k-1
// colors other than c(v), relabelled 0..K-1 by skipping c(v) and ranked by
// Eq. 1 over those labels: a sub-template table of size t keeps C(K, t-1)
// entries (the set minus c(v)), a P table of a passive child of size p keeps
// C(K, p).  In this form the eMA with a single-vertex active child is the
// identity, and every eMA and final split table is the same for all
// vertices (the plain eMA over K colors); only SpMM, which moves counts
// between vertices of different colors, re-indexes through a table keyed by
// the two colors.
//
// Layout in HBM.  Every table is vertex-major with the `batch` colorings
// interleaved innermost: element (v, I, b) sits at (v * ld + I) * batch + b
// (ld = row width padded to 16 bytes).  A vertex's row is one contiguous
// block (one gather per neighbour in SpMM), and the lanes of a warp that
// serve consecutive colorings, or consecutive (vertex, coloring) rows in the
// eMA and final step, touch consecutive addresses.  Padding entries are 0.
// The eMA and the final step see n * batch rows r = v * batch + b.
//
// FP32 tables carry a power-of-two scale per table (ScaleState): stored value
// = count * 2^-e.  Producers choose the shift from their inputs' measured
// maxima so every stored value is at most 1 and no FP32 intermediate can
// overflow; the final reduction multiplies in FP64 and applies 2^e.  FP64
// tables are unscaled exact integers while below 2^53.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "sgc_internal.h"

namespace sgc {

namespace {

constexpr int kBlock = 256;

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ float4 vadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float vmax(float4 a) { return fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)); }
__device__ __forceinline__ float vmax(double2) { return 0.f; }
template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

// SplitMix64 output number v of the stream keyed by `seed` (Steele, Lea and
// Flood 2014), high 32 bits scaled to [0, k).
__device__ __forceinline__ uint32_t vertex_color(uint64_t seed, uint32_t v, uint32_t k) {
  uint64_t z = seed + (uint64_t(v) + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (uint32_t)(((z >> 32) * (uint64_t)k) >> 32);
}

// 2^e as a float for |e| <= 126
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((127 + e) << 23);
}

// smallest s with bound * 2^-s < 1, for a finite bound >= 0
__device__ __forceinline__ int shift_for(float bound) {
  if (!(bound > 0.f)) return 0;
  return ((__float_as_int(bound) >> 23) & 0xff) - 126;
}

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ void publish_max(ScaleState* st, float m) {
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&st->max_bits, __float_as_uint(m));
}

__device__ __forceinline__ float state_max(const ScaleState* st) { return __uint_as_float(st->max_bits); }

// ------------------------------------------------------------ coloring --
__global__ void k_color(const int32_t* __restrict__ orig, int64_t n_act, int batch,
                        const uint64_t* __restrict__ seeds, int k, uint8_t* __restrict__ colors) {
  const int64_t total = n_act * batch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / batch;
    const int b = (int)(i - v * batch);
    colors[i] = (uint8_t)vertex_color(seeds[b], (uint32_t)orig[v], (uint32_t)k);
  }
}

// color word of vertex x that holds coloring b's byte (8 colorings per word)
__device__ __forceinline__ uint64_t color_word(const uint8_t* __restrict__ colors, int64_t x, int batch, int word) {
  const uint8_t* p = colors + x * batch;
  if (batch >= 8) return __ldg(reinterpret_cast<const unsigned long long*>(p) + word);
  if (batch == 4) return __ldg(reinterpret_cast<const unsigned int*>(p));
  if (batch == 2) return __ldg(reinterpret_cast<const unsigned short*>(p));
  return __ldg(p);
}

// --------------------------------------- passive single vertex: histogram --
// P(v, {d}) = number of neighbours of v with color d, for d != c(v), stored at
// the relative label of d: the SpMM of A with the one-hot leaf table
// N(u, {x}, {c}) = [c(u) = c], never materialised.  One warp per work item;
// items are the segments of heavy rows (counted with integer atomics into
// hist_heavy, by absolute color) followed by the light rows.
// The batch B is a compile-time constant: a neighbour's B color bytes come in
// one load (or B / 8 for 16 and 32 colorings) and the B counter increments are
// unrolled.
template <typename T, int B>
__global__ void k_hist(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                       const uint8_t* __restrict__ colors, int k, int32_t n_seg,
                       const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo,
                       const int32_t* __restrict__ seg_hi, int32_t n_heavy, int32_t n_act, T* __restrict__ H,
                       int64_t ldh, int32_t* __restrict__ hist_heavy, ScaleState* st_out) {
  extern __shared__ int32_t sh_hist[];
  constexpr int batch = B;
  constexpr int NW = B > 8 ? B / 8 : 1, PW = B < 8 ? B : 8;  // color words per vertex, bytes used per word
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bk = batch * k;
  int32_t* h = sh_hist + warp * bk;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  const int64_t wpb = blockDim.x >> 5;
  float wmax = 0.f;
  for (int64_t item = blockIdx.x * wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    for (int i = lane; i < bk; i += 32) h[i] = 0;
    __syncwarp();
    const bool heavy = item < n_seg;
    int32_t row, lo, hi;
    if (heavy) {
      row = seg_row[item];
      lo = seg_lo[item];
      hi = seg_hi[item];
    } else {
      row = n_heavy + (int32_t)(item - n_seg);
      lo = row_ptr[row];
      hi = row_ptr[row + 1];
    }
    for (int32_t e = lo + lane; e < hi; e += 32) {
      const int32_t u = __ldg(col_idx + e);
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint64_t x = color_word(colors, u, B, w);
#pragma unroll
        for (int i = 0; i < PW; ++i) atomicAdd(&h[(w * 8 + i) * k + (int)((x >> (8 * i)) & 0xffu)], 1);
      }
    }
    __syncwarp();
    if (heavy) {
      int32_t* dst = hist_heavy + (int64_t)row * bk;
      for (int i = lane; i < bk; i += 32)
        if (h[i]) atomicAdd(dst + i, h[i]);
    } else {
      T* out = H + (int64_t)row * batch * ldh;
      const uint8_t* cv = colors + (int64_t)row * batch;
      for (int64_t i = lane; i < batch * ldh; i += 32) {
        const int r = (int)(i / batch);
        const int b = (int)(i - (int64_t)r * batch);
        int32_t cnt = 0;
        if (r < k - 1) cnt = h[b * k + r + (r >= cv[b] ? 1 : 0)];
        out[i] = (T)cnt;
        wmax = fmaxf(wmax, (float)cnt);
      }
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, wmax);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = 0;
  }
}

template <typename T>
__global__ void k_hist_heavy_out(const int32_t* __restrict__ hist_heavy, const uint8_t* __restrict__ colors,
                                 int32_t n_heavy, int batch, int k, T* __restrict__ H, int64_t ldh,
                                 ScaleState* st_out) {
  const int64_t total = (int64_t)n_heavy * batch * ldh;
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / (ldh * batch);
    const int64_t rem = i - row * ldh * batch;
    const int r = (int)(rem / batch);
    const int64_t rb = row * batch + (rem - (int64_t)r * batch);  // row * batch + b
    int32_t cnt = 0;
    if (r < k - 1) cnt = hist_heavy[rb * k + r + (r >= colors[rb] ? 1 : 0)];
    H[i] = (T)cnt;
    m = fmaxf(m, (float)cnt);
  }
  if (std::is_same<T, float>::value) publish_max(st_out, m);
}

// -------------------------------------------------------- SpMM P = A * M --
// P(v, S) = sum over neighbours u of N(u, T_p, S), for p-subsets S without c(v).
// Neighbour u's row holds N(u, T_p, S'' + c(u)) at the relative index j of the
// (p-1)-subset S''; it contributes to v's entry for S'' + c(u) unless c(v) is
// in that set.  One warp per row (or heavy-row segment).  Lane l serves
// coloring b = l mod batch and the entries j = l / batch + L*q (L = 32 /
// batch lanes per coloring): consecutive lanes read consecutive words of the
// neighbour's row, and each lane needs one color byte of u per neighbour.
// Neighbours are accumulated in CSR order (a warp barrier separates them),
// so the summation order - and the FP32 result - is fixed.  Heavy-row
// segments write partial rows to `scratch`; k_spmm_reduce adds them in
// segment order.
//
// Two forms:
//  * direct (k_spmm): each entry is added at pos_tab[c(v)][c(u)][j] of v's row
//    (~0: dropped), accumulated in shared memory.
//  * bucketed (k_spmm_buckets, narrow rows): entries are summed into one
//    bucket row per neighbour color, Q[c(u)][j], with no lookup and no bank
//    conflict; once per row, P(v, S) = sum over the p colors c of S of
//    Q[c][index of S - c relative to c], read through inv_tab[c(v)][S].

struct SpmmItem {
  int32_t row, lo, hi;
  bool heavy;
};

__device__ __forceinline__ SpmmItem spmm_item(int64_t item, int32_t n_seg, const int32_t* __restrict__ seg_row,
                                              const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
                                              int32_t n_heavy, const int32_t* __restrict__ row_ptr) {
  SpmmItem it;
  it.heavy = item < n_seg;
  if (it.heavy) {
    it.row = seg_row[item];
    it.lo = seg_lo[item];
    it.hi = seg_hi[item];
  } else {
    it.row = n_heavy + (int32_t)(item - n_seg);
    it.lo = row_ptr[it.row];
    it.hi = row_ptr[it.row + 1];
  }
  return it;
}


// One warp per row; see the comment above for the lane mapping and the two
// forms.  NSMAX > 0: the lane's entries per neighbour (at most NSMAX) live in
// registers and the neighbour loop is software-pipelined - neighbour ids are
// fetched 32 at a time and shuffled, and the next neighbour's color word and
// row entries are loaded while the current one is added.  NSMAX = 0: plain
// loop for wide rows.
//
// The direct form's position table is either 32-bit entries read through L1
// (PT = 0; row stride w_in) or packed 1- or 2-byte entries staged in shared
// memory (PT = 1, 2; row stride tab_ld): the lanes of one coloring then read
// one shared word, so a warp's lookup touches a few banks instead of eight
// L1 lines.  All-ones entries are >= ld_out and so dropped.
template <int PT>
__device__ __forceinline__ uint32_t spmm_pos_at(const uint32_t* tab, int64_t i) {
  if (PT == 1) return reinterpret_cast<const uint8_t*>(tab)[i];
  if (PT == 2) return reinterpret_cast<const uint16_t*>(tab)[i];
  return tab[i];
}

template <typename T, bool BUCKETS, int NSMAX, int PT>
__global__ void __launch_bounds__(kBlock) k_spmm(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int batch, int k, int p,
    const T* __restrict__ Min, int w_in, int ld_in, T* __restrict__ P, int w_out, int ld_out, T* __restrict__ scratch,
    const uint32_t* __restrict__ tab_g, int tab_words_smem, int tab_ld, const ScaleState* st_in,
    ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // direct: accumulators [ld_out][batch]; bucketed: buckets [k][w_in][batch]
  const int acc_len = BUCKETS ? k * w_in * batch : ld_out * batch;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * acc_len;
  // a small index table is staged once per block after the accumulators
  const uint32_t* tab = tab_g;
  if (tab_words_smem > 0) {
    uint32_t* st = reinterpret_cast<uint32_t*>(reinterpret_cast<T*>(sm_raw) + (int64_t)wpb * acc_len);
    for (int i = threadIdx.x; i < tab_words_smem; i += blockDim.x) st[i] = __ldg(tab_g + i);
    __syncthreads();
    tab = st;
  }
  const int L = 32 / batch;
  const int b = lane & (batch - 1), jl = lane / batch;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;  // entries of this lane per neighbour
  const int64_t ld_in_row = (int64_t)batch * ld_in, ld_out_row = (int64_t)batch * ld_out;
  const int step = L * batch;  // distance between a lane's consecutive entries
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cv = (int)((color_word(colors, it.row, batch, word) >> shift) & 0xffu);
    const int cvk = cv * k;
    __syncwarp();
    if (NSMAX > 0) {
      constexpr int NU = NSMAX > 0 ? NSMAX : 1;
      for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
        const int cnt = min(32, it.hi - e0);
        const int32_t u_lane = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
        int32_t u = __shfl_sync(0xffffffffu, u_lane, 0);
        uint64_t cw = color_word(colors, u, batch, word);
        T x[NU];
        {
          const T* src = Min + (int64_t)u * ld_in_row + (int64_t)jl * batch + b;
#pragma unroll
          for (int q = 0; q < NU; ++q) x[q] = q < ns ? __ldg(src + (int64_t)step * q) : T(0);
        }
        for (int t = 0; t < cnt; ++t) {
          int32_t un = 0;
          uint64_t cwn = 0;
          T xn[NU];
          if (t + 1 < cnt) {  // prefetch the next neighbour
            un = __shfl_sync(0xffffffffu, u_lane, t + 1);
            cwn = color_word(colors, un, batch, word);
            const T* src = Min + (int64_t)un * ld_in_row + (int64_t)jl * batch + b;
#pragma unroll
            for (int q = 0; q < NU; ++q) xn[q] = q < ns ? __ldg(src + (int64_t)step * q) : T(0);
          }
          const int cu = (int)((cw >> shift) & 0xffu);
          if (BUCKETS) {
            if (cu != cv) {  // a neighbour of v's own color never contributes
              T* qrow = acc + (cu * w_in + jl) * batch + b;
#pragma unroll
              for (int q = 0; q < NU; ++q)
                if (q < ns) qrow[step * q] += x[q];
            }
          } else {
            const int64_t pt = (int64_t)(cvk + cu) * tab_ld + jl;
            uint32_t pos[NU];
#pragma unroll
            for (int q = 0; q < NU; ++q) pos[q] = q < ns ? spmm_pos_at<PT>(tab, pt + L * q) : 0xFFFFFFFFu;
#pragma unroll
            for (int q = 0; q < NU; ++q)
              if (pos[q] < (uint32_t)ld_out) acc[pos[q] * batch + b] += x[q];
          }
          __syncwarp();
          cw = cwn;
#pragma unroll
          for (int q = 0; q < NU; ++q) x[q] = xn[q];
        }
      }
    } else {
      for (int32_t e = it.lo; e < it.hi; ++e) {
        const int32_t u = __ldg(col_idx + e);
        const int cu = (int)((color_word(colors, u, batch, word) >> shift) & 0xffu);
        const T* src = Min + (int64_t)u * ld_in_row + (int64_t)jl * batch + b;
        if (BUCKETS) {
          if (cu != cv) {
            T* qrow = acc + (cu * w_in + jl) * batch + b;
            for (int q = 0; q < ns; ++q) qrow[step * q] += __ldg(src + (int64_t)step * q);
          }
        } else {
          const int64_t pt = (int64_t)(cvk + cu) * tab_ld + jl;
          int q = 0;
          for (; q + 4 <= ns; q += 4) {
            // the gathers do not wait for the positions (memory-level parallelism)
            const uint32_t p0 = spmm_pos_at<PT>(tab, pt + L * q), p1 = spmm_pos_at<PT>(tab, pt + L * (q + 1));
            const uint32_t p2 = spmm_pos_at<PT>(tab, pt + L * (q + 2)), p3 = spmm_pos_at<PT>(tab, pt + L * (q + 3));
            const T x0 = __ldg(src + (int64_t)step * q), x1 = __ldg(src + (int64_t)step * (q + 1));
            const T x2 = __ldg(src + (int64_t)step * (q + 2)), x3 = __ldg(src + (int64_t)step * (q + 3));
            if (p0 < (uint32_t)ld_out) acc[p0 * batch + b] += x0;
            if (p1 < (uint32_t)ld_out) acc[p1 * batch + b] += x1;
            if (p2 < (uint32_t)ld_out) acc[p2 * batch + b] += x2;
            if (p3 < (uint32_t)ld_out) acc[p3 * batch + b] += x3;
          }
          for (; q < ns; ++q) {
            const uint32_t p0 = spmm_pos_at<PT>(tab, pt + L * q);
            if (p0 < (uint32_t)ld_out) acc[p0 * batch + b] += __ldg(src + (int64_t)step * q);
          }
        }
        __syncwarp();
      }
    }
    T* dst = it.heavy ? scratch + item * ld_out_row : P + (int64_t)it.row * ld_out_row;
    if (BUCKETS) {
      // resolve: P(v, S) = sum over the colors c of S of Q[c][index of S - c relative to c]
      for (int i = lane; i < ld_out * batch; i += 32) {
        const int S = i / batch, bb = i - S * batch;
        T val = T(0);
        if (S < w_out) {
          const int cvb = (int)((color_word(colors, it.row, batch, bb >> 3) >> ((bb & 7) * 8)) & 0xffu);
          const uint32_t* ent = tab + ((int64_t)cvb * w_out + S) * p;
          for (int t = 0; t < p; ++t) {
            const uint32_t e = ent[t];
            const int c = (int)(e & 0xffu), j = (int)(e >> 8);
            if (c < k && j < w_in) val += acc[(c * w_in + j) * batch + bb];
          }
        }
        dst[i] = val;
        if (!it.heavy) m = fmaxf(m, (float)val);
      }
    } else {
      for (int i = lane; i < acc_len; i += 32) {
        const T x = acc[i];
        dst[i] = x;
        if (!it.heavy) m = fmaxf(m, (float)x);
      }
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Direct form with the next neighbour's id and color word fetched one step
// ahead and all of a neighbour's position and row loads issued together
// (at most NSMAX per lane, unrolled), so each neighbour costs about one memory
// latency.  Same results and summation order as k_spmm's direct form.
template <typename T, int NSMAX>
__global__ void __launch_bounds__(kBlock) k_spmm_direct_pf(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int batch, int k,
    const T* __restrict__ Min, int w_in, int ld_in, T* __restrict__ P, int ld_out, T* __restrict__ scratch,
    const uint32_t* __restrict__ tab, const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int acc_len = ld_out * batch;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * acc_len;
  const int L = 32 / batch;
  const int b = lane & (batch - 1), jl = lane / batch;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;
  const int64_t ld_in_row = (int64_t)batch * ld_in, ld_out_row = (int64_t)batch * ld_out;
  const int step = L * batch;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cvk = (int)((color_word(colors, it.row, batch, word) >> shift) & 0xffu) * k;
    __syncwarp();
    int32_t u_n = it.lo < it.hi ? __ldg(col_idx + it.lo) : 0;
    uint64_t cw_n = color_word(colors, u_n, batch, word);
    for (int32_t e = it.lo; e < it.hi; ++e) {
      const int32_t u = u_n;
      const uint64_t cw = cw_n;
      if (e + 1 < it.hi) {
        u_n = __ldg(col_idx + e + 1);
        cw_n = color_word(colors, u_n, batch, word);
      }
      const int cu = (int)((cw >> shift) & 0xffu);
      const uint32_t* pt = tab + (int64_t)(cvk + cu) * w_in + jl;
      const T* src = Min + (int64_t)u * ld_in_row + (int64_t)jl * batch + b;
      uint32_t pos[NSMAX];
      T x[NSMAX];
#pragma unroll
      for (int q = 0; q < NSMAX; ++q) {
        pos[q] = q < ns ? pt[L * q] : 0xFFFFFFFFu;
        x[q] = q < ns ? __ldg(src + (int64_t)step * q) : T(0);
      }
#pragma unroll
      for (int q = 0; q < NSMAX; ++q)
        if (pos[q] < (uint32_t)ld_out) acc[pos[q] * batch + b] += x[q];
      __syncwarp();
    }
    T* dst = it.heavy ? scratch + item * ld_out_row : P + (int64_t)it.row * ld_out_row;
    for (int i = lane; i < acc_len; i += 32) {
      const T x = acc[i];
      dst[i] = x;
      if (!it.heavy) m = fmaxf(m, (float)x);
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Direct form with the batch B as a compile-time constant.  Lane l serves
// coloring l % B and the entries j = l / B + (32 / B) q, which sit at
// row[l + 32 q] of the neighbour's interleaved row, so the gathers and the
// accumulator addresses are immediate offsets from per-neighbour bases.  The
// position table is either the 32-bit [c_v][c_u][j] one (LM = false) or
// lane-major with 16-bit entries (tab16[c_v][c_u][jl][q], nsp entries per
// lane, all ones = nowhere), from which a lane reads four positions with one
// 8-byte load (LM = true; faster for some widths and batches, slower for
// others: the autotuner picks).  G > 0 issues G predicated entries per lane at
// once (more loads in flight for wide rows); G = 0 takes four at a time.  Neighbour ids and their color words are read
// 32 at a time, one per lane, and shuffled.  Same summation order as k_spmm's
// direct form.
//
// PRIV: every lane accumulates into its own shared-memory column
// (acc[pos * 32 + lane], one bank per lane), so the scattered adds never
// conflict; the L = 32 / B partial rows of a coloring are summed with warp
// shuffles when the row is written (L * 32 * ld_out entries of shared memory
// per warp instead of B * ld_out).
template <typename T, int B, bool LM, int G, bool PRIV = false>
__global__ void __launch_bounds__(kBlock) k_spmm_d(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int k, const T* __restrict__ Min, int w_in,
    int ld_in, T* __restrict__ P, int ld_out, T* __restrict__ scratch, const uint32_t* __restrict__ tab, int nsp,
    const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int L = 32 / B;
  constexpr int NW = B > 8 ? B / 8 : 1;  // color words per vertex
  constexpr int AS = PRIV ? 32 : B;       // accumulator entries per position
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int acc_len = ld_out * AS;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * acc_len;
  const int ab = PRIV ? lane : lane % B;  // this lane's accumulator column
  const int b = lane % B, jl = lane / B;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;
  const int64_t row_len = (int64_t)ld_in * B;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  const uint16_t* tab16 = reinterpret_cast<const uint16_t*>(tab);
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cvk = (int)((color_word(colors, it.row, B, word) >> shift) & 0xffu) * k;
    __syncwarp();
    for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
      const int cnt = min(32, it.hi - e0);
      const int32_t u_lane = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
      uint64_t w_lane[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) w_lane[w] = color_word(colors, u_lane, B, w);
      for (int t = 0; t < cnt; ++t) {
        const int32_t u = __shfl_sync(0xffffffffu, u_lane, t);
        uint64_t cw = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint64_t x = __shfl_sync(0xffffffffu, w_lane[w], t);
          if (w == word) cw = x;
        }
        const int cu = (int)((cw >> shift) & 0xffu);
        const T* src = Min + (int64_t)u * row_len + lane;
        if (LM) {  // lane-major 16-bit table: four positions per load
          const uint16_t* pt = tab16 + ((int64_t)(cvk + cu) * L + jl) * nsp;
          for (int q = 0; q < ns; q += 4) {
            const uint2 pv = __ldg(reinterpret_cast<const uint2*>(pt + q));
            const uint32_t p0 = pv.x & 0xffffu, p1 = pv.x >> 16, p2 = pv.y & 0xffffu, p3 = pv.y >> 16;
            const T x0 = __ldg(src + 32 * q);
            const T x1 = q + 1 < ns ? __ldg(src + 32 * (q + 1)) : T(0);
            const T x2 = q + 2 < ns ? __ldg(src + 32 * (q + 2)) : T(0);
            const T x3 = q + 3 < ns ? __ldg(src + 32 * (q + 3)) : T(0);
            if (p0 < (uint32_t)ld_out) acc[p0 * AS + ab] += x0;
            if (p1 < (uint32_t)ld_out) acc[p1 * AS + ab] += x1;
            if (p2 < (uint32_t)ld_out) acc[p2 * AS + ab] += x2;
            if (p3 < (uint32_t)ld_out) acc[p3 * AS + ab] += x3;
          }
        } else if (G == 0) {  // 32-bit table [c_v][c_u][j], four entries at a time
          const uint32_t* pt = tab + (cvk + cu) * w_in + jl;
          int q = 0;
          for (; q + 4 <= ns; q += 4) {
            const uint32_t p0 = pt[L * q], p1 = pt[L * (q + 1)], p2 = pt[L * (q + 2)], p3 = pt[L * (q + 3)];
            const T x0 = __ldg(src + 32 * q), x1 = __ldg(src + 32 * (q + 1));
            const T x2 = __ldg(src + 32 * (q + 2)), x3 = __ldg(src + 32 * (q + 3));
            if (p0 < (uint32_t)ld_out) acc[p0 * AS + ab] += x0;
            if (p1 < (uint32_t)ld_out) acc[p1 * AS + ab] += x1;
            if (p2 < (uint32_t)ld_out) acc[p2 * AS + ab] += x2;
            if (p3 < (uint32_t)ld_out) acc[p3 * AS + ab] += x3;
          }
          for (; q < ns; ++q) {
            const uint32_t p0 = pt[L * q];
            const T x0 = __ldg(src + 32 * q);
            if (p0 < (uint32_t)ld_out) acc[p0 * AS + ab] += x0;
          }
        } else {  // 32-bit table, G entries per lane in flight at once (predicated)
          constexpr int GG = G > 0 ? G : 1;
          const uint32_t* pt = tab + (cvk + cu) * w_in + jl;
          for (int q = 0; q < ns; q += GG) {
            uint32_t pp[GG];
            T xx[GG];
#pragma unroll
            for (int i = 0; i < GG; ++i) {
              const bool ok = q + i < ns;
              pp[i] = ok ? pt[L * (q + i)] : 0xFFFFFFFFu;
              xx[i] = ok ? __ldg(src + 32 * (q + i)) : T(0);
            }
#pragma unroll
            for (int i = 0; i < GG; ++i)
              if (pp[i] < (uint32_t)ld_out) acc[pp[i] * AS + ab] += xx[i];
          }
        }
        __syncwarp();
      }
    }
    const int out_len = ld_out * B;
    T* dst = it.heavy ? scratch + item * (int64_t)out_len : P + (int64_t)it.row * out_len;
    if (PRIV) {
      // positions g*L .. g*L+L-1: lane (jl, b) ends up holding position g*L + jl of coloring b
      // summed over the L partial columns, and writes dst[g * 32 + lane] (coalesced)
      __syncwarp();
      for (int g = 0; g * L < ld_out; ++g) {
        T mine = T(0);
#pragma unroll
        for (int r = 0; r < L; ++r) {
          T v = g * L + r < ld_out ? acc[(g * L + r) * 32 + lane] : T(0);
#pragma unroll
          for (int o = B; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (r == jl) mine = v;
        }
        if (g * L + jl < ld_out) {
          dst[g * 32 + lane] = mine;
          if (!it.heavy) m = fmaxf(m, (float)mine);
        }
      }
    } else {
      for (int i = lane; i < acc_len; i += 32) {
        const T x = acc[i];
        dst[i] = x;
        if (!it.heavy) m = fmaxf(m, (float)x);
      }
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Direct form, unrolled: the batch B and a bound NS on a lane's entries per
// neighbour (ns <= NS <= 16) are compile-time constants.  The lane's positions
// for a neighbour come in one 16-byte load - 8-bit entries, byte q for entry
// j = jl + L q of the (c_v, c_u) pair, 0xFF = dropped (table OP_SPMM + 600) -
// instead of one 32-bit lookup per entry through L1, and the next neighbour's
// id, color, positions and row entries are loaded while the current one is
// added.  Same summation order as k_spmm_d (a warp barrier between
// neighbours; a position receives at most one term per neighbour).
template <typename T, int B, int NS>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 8 && NS > 9 ? 4 : 5) k_spmm_u(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int k, const T* __restrict__ Min, int w_in,
    int ld_in, T* __restrict__ P, int ld_out, T* __restrict__ scratch, const uint4* __restrict__ tab,
    const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int L = 32 / B;
  constexpr int NW = B > 8 ? B / 8 : 1;  // color words per vertex
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int acc_len = ld_out * B;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * acc_len;
  const int b = lane % B, jl = lane / B;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;
  const int64_t row_len = (int64_t)ld_in * B;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cvk = (int)((color_word(colors, it.row, B, word) >> shift) & 0xffu) * k;
    __syncwarp();
    for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
      const int cnt = min(32, it.hi - e0);
      const int32_t u_lane = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
      uint64_t w_lane[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) w_lane[w] = color_word(colors, u_lane, B, w);
      // neighbour t's positions and entries (loaded one neighbour ahead)
      auto fetch = [&](int t, uint4& pw, T (&x)[NS]) {
        const int32_t u = __shfl_sync(0xffffffffu, u_lane, t);
        uint64_t cw = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint64_t y = __shfl_sync(0xffffffffu, w_lane[w], t);
          if (w == word) cw = y;
        }
        const int cu = (int)((cw >> shift) & 0xffu);
        pw = __ldg(tab + (int64_t)(cvk + cu) * L + jl);
        const T* src = Min + (int64_t)u * row_len + lane;
#pragma unroll
        for (int q = 0; q < NS; ++q) x[q] = q < ns ? __ldg(src + 32 * q) : T(0);
      };
      auto add = [&](const uint4& pw, const T (&x)[NS]) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          const uint32_t wq = q < 4 ? pw.x : q < 8 ? pw.y : q < 12 ? pw.z : pw.w;
          const uint32_t p = (wq >> (8 * (q & 3))) & 0xffu;
          if (p < (uint32_t)ld_out) acc[p * B + b] += x[q];
        }
        __syncwarp();
      };
      if (NS <= 4) {  // few entries per lane: keep the next neighbour's loads in flight too
        uint4 pw;
        T x[NS];
        fetch(0, pw, x);
        for (int t = 0; t < cnt; ++t) {
          uint4 pn = pw;
          T xn[NS];
#pragma unroll
          for (int q = 0; q < NS; ++q) xn[q] = T(0);
          if (t + 1 < cnt) fetch(t + 1, pn, xn);
          add(pw, x);
          pw = pn;
#pragma unroll
          for (int q = 0; q < NS; ++q) x[q] = xn[q];
        }
      } else {  // NS loads per lane already in flight per neighbour
        for (int t = 0; t < cnt; ++t) {
          uint4 pw;
          T x[NS];
          fetch(t, pw, x);
          add(pw, x);
        }
      }
    }
    const int out_len = ld_out * B;
    T* dst = it.heavy ? scratch + item * (int64_t)out_len : P + (int64_t)it.row * out_len;
    for (int i = lane; i < acc_len; i += 32) {
      const T v = acc[i];
      dst[i] = v;
      if (!it.heavy) m = fmaxf(m, (float)v);
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Direct form for wide rows: like k_spmm_u, but with 16-bit positions in
// chunks of eight - one 16-byte load per lane, neighbour and eight entries
// (table OP_SPMM + 700: for each (c_v, c_u) pair and lane position jl, nch
// chunks; 0xFFFF = dropped) - and a runtime chunk count, so any row width
// works; the row entries of two chunks are loaded together.  Same summation
// order as k_spmm_d.
template <typename T, int B>
__global__ void __launch_bounds__(kBlock) k_spmm_w(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int k, const T* __restrict__ Min, int w_in,
    int ld_in, T* __restrict__ P, int ld_out, T* __restrict__ scratch, const uint4* __restrict__ tab,
    const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int L = 32 / B;
  constexpr int NW = B > 8 ? B / 8 : 1;  // color words per vertex
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int acc_len = ld_out * B;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * acc_len;
  const int b = lane % B, jl = lane / B;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;
  const int nch = ((w_in + L - 1) / L + 7) / 8;  // chunks per lane (the same for every lane)
  const int64_t row_len = (int64_t)ld_in * B;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cvk = (int)((color_word(colors, it.row, B, word) >> shift) & 0xffu) * k;
    __syncwarp();
    for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
      const int cnt = min(32, it.hi - e0);
      const int32_t u_lane = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
      uint64_t w_lane[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) w_lane[w] = color_word(colors, u_lane, B, w);
      for (int t = 0; t < cnt; ++t) {
        const int32_t u = __shfl_sync(0xffffffffu, u_lane, t);
        uint64_t cw = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint64_t y = __shfl_sync(0xffffffffu, w_lane[w], t);
          if (w == word) cw = y;
        }
        const int cu = (int)((cw >> shift) & 0xffu);
        const uint4* pt = tab + ((int64_t)(cvk + cu) * L + jl) * nch;
        const T* src = Min + (int64_t)u * row_len + lane;
        // two chunks (16 entries) per step: sixteen row loads in flight per lane
        for (int c = 0; c < nch; c += 2) {
          const uint4 pa = __ldg(pt + c);
          const uint4 pb = c + 1 < nch ? __ldg(pt + c + 1) : make_uint4(~0u, ~0u, ~0u, ~0u);
          T x[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int q = 8 * c + i;
            x[i] = q < ns ? __ldg(src + 32 * q) : T(0);
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const uint4& pw = i < 8 ? pa : pb;
            const int ii = i & 7;
            const uint32_t wq = ii < 2 ? pw.x : ii < 4 ? pw.y : ii < 6 ? pw.z : pw.w;
            const uint32_t p = (wq >> (16 * (ii & 1))) & 0xffffu;
            if (p < (uint32_t)ld_out) acc[p * B + b] += x[i];
          }
        }
        __syncwarp();
      }
    }
    const int out_len = ld_out * B;
    T* dst = it.heavy ? scratch + item * (int64_t)out_len : P + (int64_t)it.row * out_len;
    for (int i = lane; i < acc_len; i += 32) {
      const T v = acc[i];
      dst[i] = v;
      if (!it.heavy) m = fmaxf(m, (float)v);
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Bucketed form with the batch B as a compile-time constant: a lane's entries
// of a neighbour's row are row[l + 32 q] and land in bucket row
// Q[c(u)][l + 32 q] (no lookup, conflict-free), neighbour ids and color words
// are shuffled from one load per 32 neighbours, and in the resolve step a
// lane only ever serves its own coloring (B divides 32), so v's color is the
// one already in a register.  The resolve table is staged in shared memory
// when small (tab_words_smem words).  Same sums, in the same order, as
// k_spmm's bucketed form.
template <typename T, int B>
__global__ void __launch_bounds__(kBlock) k_spmm_bk(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int k, int p, const T* __restrict__ Min,
    int w_in, int ld_in, T* __restrict__ P, int w_out, int ld_out, T* __restrict__ scratch,
    const uint32_t* __restrict__ tab_g, int tab_words_smem, const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int L = 32 / B;
  constexpr int NW = B > 8 ? B / 8 : 1;
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int acc_len = k * w_in * B;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * acc_len;
  const uint32_t* tab = tab_g;
  if (tab_words_smem > 0) {
    uint32_t* stab = reinterpret_cast<uint32_t*>(reinterpret_cast<T*>(sm_raw) + (int64_t)wpb * acc_len);
    for (int i = threadIdx.x; i < tab_words_smem; i += blockDim.x) stab[i] = __ldg(tab_g + i);
    __syncthreads();
    tab = stab;
  }
  const int b = lane % B, jl = lane / B;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;
  const int64_t row_len = (int64_t)ld_in * B;
  const int bucket_len = w_in * B;
  const int out_len = ld_out * B;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cv = (int)((color_word(colors, it.row, B, word) >> shift) & 0xffu);
    __syncwarp();
    for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
      const int cnt = min(32, it.hi - e0);
      const int32_t u_lane = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
      uint64_t w_lane[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) w_lane[w] = color_word(colors, u_lane, B, w);
      for (int t = 0; t < cnt; ++t) {
        const int32_t u = __shfl_sync(0xffffffffu, u_lane, t);
        uint64_t cw = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint64_t x = __shfl_sync(0xffffffffu, w_lane[w], t);
          if (w == word) cw = x;
        }
        const int cu = (int)((cw >> shift) & 0xffu);
        if (cu != cv) {  // a neighbour of v's own color never contributes
          T* qrow = acc + cu * bucket_len + lane;
          const T* src = Min + (int64_t)u * row_len + lane;
          int q = 0;
          for (; q + 4 <= ns; q += 4) {
            const T x0 = __ldg(src + 32 * q), x1 = __ldg(src + 32 * (q + 1));
            const T x2 = __ldg(src + 32 * (q + 2)), x3 = __ldg(src + 32 * (q + 3));
            qrow[32 * q] += x0;
            qrow[32 * (q + 1)] += x1;
            qrow[32 * (q + 2)] += x2;
            qrow[32 * (q + 3)] += x3;
          }
          for (; q < ns; ++q) qrow[32 * q] += __ldg(src + 32 * q);
        }
        __syncwarp();
      }
    }
    // resolve: P(v, S) = sum over the colors c of S of Q[c][index of S - c relative to c]
    T* dst = it.heavy ? scratch + item * (int64_t)out_len : P + (int64_t)it.row * out_len;
    const uint32_t* ent0 = tab + (int64_t)cv * w_out * p;
    for (int i = lane; i < out_len; i += 32) {
      const int S = i / B;
      T val = T(0);
      if (S < w_out) {
        const uint32_t* ent = ent0 + (int64_t)S * p;
        for (int t = 0; t < p; ++t) {
          const uint32_t e = ent[t];
          const int c = (int)(e & 0xffu), j = (int)(e >> 8);
          if (c < k && j < w_in) val += acc[(c * w_in + j) * B + b];
        }
      }
      dst[i] = val;
      if (!it.heavy) m = fmaxf(m, (float)val);
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Direct form with the neighbour rows streamed into shared memory by
// asynchronous copies (cp.async, 16 bytes per lane), R neighbours ahead of the
// one being added: a warp keeps R rows (and their color bytes) in flight
// without holding them in registers, so the gathers' latency overlaps the
// adds.  Each ring slot holds a neighbour's `batch` color bytes (hdr bytes,
// 16-byte aligned) and then its whole interleaved row (ld_in * batch entries).
// Neighbour ids are read 32 at a time, one chunk ahead.  Same summation order
// as k_spmm's direct form.  batch >= 4 (the color bytes are one 4-, 8- or
// 16-byte copy, or two for 32 colorings).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T, int R>
__global__ void __launch_bounds__(kBlock) k_spmm_ring(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int batch, int k,
    const T* __restrict__ Min, int w_in, int ld_in, T* __restrict__ P, int ld_out, T* __restrict__ scratch,
    const uint32_t* __restrict__ tab, const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int acc_len = ld_out * batch;
  const int hdr = batch < 16 ? 16 : batch;                          // color bytes, padded
  const int row_bytes = ld_in * batch * (int)sizeof(T);             // a multiple of 16
  const int slot_bytes = hdr + row_bytes;
  const int warp_bytes = ((acc_len * (int)sizeof(T) + 15) & ~15) + R * slot_bytes;
  unsigned char* wbase = sm_raw + (int64_t)warp * warp_bytes;
  T* acc = reinterpret_cast<T*>(wbase);
  unsigned char* ring = wbase + ((acc_len * (int)sizeof(T) + 15) & ~15);
  const int L = 32 / batch;
  const int b = lane & (batch - 1), jl = lane / batch;
  const int word = b >> 3, shift = (b & 7) * 8;
  const int ns = jl < w_in ? (w_in - jl + L - 1) / L : 0;
  const int n16 = row_bytes >> 4;
  const int64_t ld_out_row = (int64_t)batch * ld_out;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  const unsigned char* Mb = reinterpret_cast<const unsigned char*>(Min);
  // issue the copies of neighbour u into ring slot `sl` (all lanes take part)
  auto issue = [&](int sl, int32_t u) {
    unsigned char* dst = ring + sl * slot_bytes;
    const unsigned char* crow = colors + (int64_t)u * batch;
    if (lane == 0) {
      if (batch == 4) cp_async_small<4>(dst, crow);
      else if (batch == 8) cp_async_small<8>(dst, crow);
      else cp_async16(dst, crow);
    } else if (lane == 1 && batch == 32) {
      cp_async16(dst + 16, crow + 16);
    }
    const unsigned char* src = Mb + (int64_t)u * row_bytes;
    for (int c = lane; c < n16; c += 32) cp_async16(dst + hdr + c * 16, src + c * 16);
  };
  float m = 0.f;
  for (int64_t item = blockIdx.x * (int64_t)wpb + warp; item < nitems; item += (int64_t)gridDim.x * wpb) {
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    for (int i = lane; i < acc_len; i += 32) acc[i] = T(0);
    const int cvk = (int)((color_word(colors, it.row, batch, word) >> shift) & 0xffu) * k;
    const int deg = it.hi - it.lo;
    int32_t ids_cur = lane < deg ? __ldg(col_idx + it.lo + lane) : 0;
    int32_t ids_nxt = 32 + lane < deg ? __ldg(col_idx + it.lo + 32 + lane) : 0;
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const int32_t u = __shfl_sync(0xffffffffu, ids_cur, s);
      if (s < deg) issue(s, u);
      cp_async_commit();
    }
    for (int i = 0; i < deg; ++i) {
      if (i > 0 && (i & 31) == 0) {  // next chunk of neighbour ids
        ids_cur = ids_nxt;
        ids_nxt = i + 32 + lane < deg ? __ldg(col_idx + it.lo + i + 32 + lane) : 0;
      }
      cp_async_wait<R - 1>();
      __syncwarp();
      const unsigned char* slot = ring + (i % R) * slot_bytes;
      const int cu = slot[b];
      const T* row = reinterpret_cast<const T*>(slot + hdr);
      const uint32_t* pt = tab + (int64_t)(cvk + cu) * w_in + jl;
      int q = 0;
      for (; q + 4 <= ns; q += 4) {
        const uint32_t p0 = pt[L * q], p1 = pt[L * (q + 1)];
        const uint32_t p2 = pt[L * (q + 2)], p3 = pt[L * (q + 3)];
        const T x0 = row[lane + 32 * q], x1 = row[lane + 32 * (q + 1)];
        const T x2 = row[lane + 32 * (q + 2)], x3 = row[lane + 32 * (q + 3)];
        if (p0 < (uint32_t)ld_out) acc[p0 * batch + b] += x0;
        if (p1 < (uint32_t)ld_out) acc[p1 * batch + b] += x1;
        if (p2 < (uint32_t)ld_out) acc[p2 * batch + b] += x2;
        if (p3 < (uint32_t)ld_out) acc[p3 * batch + b] += x3;
      }
      for (; q < ns; ++q) {
        const uint32_t p0 = pt[L * q];
        if (p0 < (uint32_t)ld_out) acc[p0 * batch + b] += row[lane + 32 * q];
      }
      __syncwarp();  // every lane is done with this slot before it is refilled
      const int nx = i + R;  // the neighbour whose row goes into this slot next
      const int32_t u = __shfl_sync(0xffffffffu, (nx & ~31) == (i & ~31) ? ids_cur : ids_nxt, nx & 31);
      if (nx < deg) issue(i % R, u);
      cp_async_commit();
    }
    T* dst = it.heavy ? scratch + item * ld_out_row : P + (int64_t)it.row * ld_out_row;
    __syncwarp();
    for (int i = lane; i < acc_len; i += 32) {
      const T x = acc[i];
      dst[i] = x;
      if (!it.heavy) m = fmaxf(m, (float)x);
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Register-bucket form, for passes of one coloring (batch 1).  All 32 lanes of
// a warp work on the same row and coloring, so a neighbour's color c(u) is the
// same for the whole warp: its row entries are added to the register bucket
// Q[c(u)] through a warp-uniform switch - no index lookup and no shared-memory
// traffic per neighbour, only the coalesced gather.  A row's w_in columns are
// split over `wpr` warps of 32 * NS columns; the buckets are then flushed to
// shared memory and P(v, S) = sum over the colors c of S of Q[c][S - c]
// resolved through inv_tab[c(v)][S] as in the bucketed form.  Neighbours are
// added in CSR order (fixed FP32 summation order).
#define SGC_RB_CASE(C)                               \
  case C:                                            \
    _Pragma("unroll") for (int q = 0; q < NS; ++q) { \
      acc[C][q] += x[i][q];                          \
    }                                                \
    break;

template <typename T, int NS>
__global__ void __launch_bounds__(kBlock) k_spmm_rb(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int k, int p, const T* __restrict__ Min,
    int w_in, int ld_in, T* __restrict__ P, int w_out, int ld_out, T* __restrict__ scratch,
    const uint32_t* __restrict__ inv_tab, int wpr, const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int UNR = 4;  // neighbours whose loads are in flight together
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = (blockDim.x >> 5) / wpr;  // row slots per block
  const int slot = warp / wpr, slice = warp - slot * wpr;
  const int qlen = k * w_in;
  T* Qs = reinterpret_cast<T*>(sm_raw) + (int64_t)slot * qlen;
  const int j0 = slice * 32 * NS + lane;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t base = (int64_t)blockIdx.x * rows; base < nitems; base += (int64_t)gridDim.x * rows) {
    const int64_t item = base + slot;
    const bool valid = item < nitems;
    SpmmItem it{0, 0, 0, false};
    int cv = 0;
    if (valid) {
      it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
      cv = __ldg(colors + it.row);
      T acc[16][NS];
#pragma unroll
      for (int c = 0; c < 16; ++c)
#pragma unroll
        for (int q = 0; q < NS; ++q) acc[c][q] = T(0);
      for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
        const int cnt = min(32, it.hi - e0);
        const int32_t u_lane = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
        const int c_lane = lane < cnt ? (int)__ldg(colors + u_lane) : cv;
        for (int t = 0; t < cnt; t += UNR) {
          T x[UNR][NS];
          int cu[UNR];
#pragma unroll
          for (int i = 0; i < UNR; ++i) {
            const int tt = t + i;
            const int32_t u = __shfl_sync(0xffffffffu, u_lane, tt & 31);
            cu[i] = __shfl_sync(0xffffffffu, c_lane, tt & 31);
            if (tt >= cnt) cu[i] = cv;  // past the chunk: contributes nothing
            const T* src = Min + (int64_t)u * ld_in;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
              const int j = j0 + 32 * q;
              x[i][q] = (tt < cnt && j < w_in) ? __ldg(src + j) : T(0);
            }
          }
#pragma unroll
          for (int i = 0; i < UNR; ++i) {
            if (cu[i] == cv) continue;  // a neighbour of v's own color never contributes
            switch (cu[i]) {
              SGC_RB_CASE(0) SGC_RB_CASE(1) SGC_RB_CASE(2) SGC_RB_CASE(3)
              SGC_RB_CASE(4) SGC_RB_CASE(5) SGC_RB_CASE(6) SGC_RB_CASE(7)
              SGC_RB_CASE(8) SGC_RB_CASE(9) SGC_RB_CASE(10) SGC_RB_CASE(11)
              SGC_RB_CASE(12) SGC_RB_CASE(13) SGC_RB_CASE(14) SGC_RB_CASE(15)
              default: break;
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < k) {
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            const int j = j0 + 32 * q;
            if (j < w_in) Qs[c * w_in + j] = acc[c][q];
          }
        }
    }
    __syncthreads();
    if (valid) {
      T* dst = it.heavy ? scratch + item * (int64_t)ld_out : P + (int64_t)it.row * ld_out;
      const uint32_t* ent0 = inv_tab + (int64_t)cv * w_out * p;
      for (int i = slice * 32 + lane; i < ld_out; i += wpr * 32) {
        T val = T(0);
        if (i < w_out) {
          const uint32_t* ent = ent0 + (int64_t)i * p;
          for (int t = 0; t < p; ++t) {
            const uint32_t e = __ldg(ent + t);
            const int c = (int)(e & 0xffu), j = (int)(e >> 8);
            if (c < k && j < w_in) val += Qs[c * w_in + j];
          }
        }
        dst[i] = val;
        if (!it.heavy) m = fmaxf(m, (float)val);
      }
    }
    __syncthreads();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}
#undef SGC_RB_CASE

// heavy rows: P(h, :) = sum of the row's segment partials, in segment order
template <typename T>
__global__ void k_spmm_reduce(const int32_t* __restrict__ heavy_seg, int32_t n_heavy, const T* __restrict__ scratch,
                              int64_t width, T* __restrict__ P, int64_t ld_row, ScaleState* st_out) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  const int64_t wv = width / VN;
  const int64_t total = (int64_t)n_heavy * wv;
  const V* S = reinterpret_cast<const V*>(scratch);
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t h = i / wv, cv = i - h * wv;
    V acc = vzero<V>();
    for (int32_t s = heavy_seg[h]; s < heavy_seg[h + 1]; ++s) acc = vadd(acc, S[(int64_t)s * wv + cv]);
    reinterpret_cast<V*>(P)[h * (ld_row / VN) + cv] = acc;
    m = fmaxf(m, vmax(acc));
  }
  if (std::is_same<T, float>::value) publish_max(st_out, m);
}

// The pruned neighbour sums one passive column at a time (the ablation of the
// SpMM's row-wise vectorisation): P(v, S) for one column S, then the next -
// a thread per (column S, row r = (v, coloring)), columns outermost, walks v's
// whole neighbour list and adds the one entry of each neighbour's row that
// holds S (index npos[c_v][S][c_u], ~0 when c_u is not in S).  Every P entry is
// computed once, as in the pruned method, but each neighbour visit reads a
// single entry instead of the neighbour's row.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_spmm_col(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_act,
    const uint8_t* __restrict__ colors, int lb, int k, const T* __restrict__ Mp, int64_t ldp, T* __restrict__ P,
    int64_t ld_out, int w_out, const uint32_t* __restrict__ npos, const ScaleState* st_in, ScaleState* st_out) {
  const int64_t rows = (int64_t)n_act << lb;
  const int64_t items = rows * ld_out;
  const int batch = 1 << lb;
  float m = 0.f;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int S = (int)(it / rows);
    const int64_t r = it - (int64_t)S * rows;
    const int64_t v = r >> lb;
    const int b = (int)(r & (batch - 1));
    T sum = T(0);
    if (S < w_out) {
      const uint32_t* np = npos + ((int64_t)colors[r] * w_out + S) * k;
      for (int32_t q = row_ptr[v]; q < row_ptr[v + 1]; ++q) {
        const int32_t u = __ldg(col_idx + q);
        const uint32_t pj = __ldg(np + colors[(int64_t)u * batch + b]);
        if (pj != 0xFFFFFFFFu) sum += __ldg(Mp + (((int64_t)u * ldp + pj) << lb) + b);
      }
    }
    P[((v * ld_out + S) << lb) + b] = sum;
    m = fmaxf(m, (float)sum);
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// ---------------------------------------------- neighbours grouped by color --
// For the grouped SpMM form, per coloring b: the neighbours u of a row (or a
// heavy-row segment) whose color differs from the row's, grouped by color in
// ascending order and in CSR order within a color, at ids[b * nnz + lo + i]
// and cols[b * nnz + lo + i] for i < kept[item * B + b] (lo = the item's first
// entry).  Neighbours of the row's own color are dropped: every set they hold
// contains c(v), and v's P row keeps no such set.  A warp per (item,
// coloring) does a two-pass counting sort of its at most 256 entries (longer
// rows are cut into segments); colors are below 32.
template <int B>
__global__ void __launch_bounds__(kBlock) k_group_nbrs(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_seg,
    const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi,
    int32_t n_heavy, int32_t n_act, const uint8_t* __restrict__ colors, int64_t nnz, int32_t* __restrict__ gids,
    uint8_t* __restrict__ gcols, int32_t* __restrict__ gkept) {
  __shared__ int cnt_sm[kBlock / 32][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  int* cnt = cnt_sm[warp];
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  for (int64_t w = blockIdx.x * (int64_t)wpb + warp; w < nitems * B; w += (int64_t)gridDim.x * wpb) {
    const int64_t item = w / B;
    const int b = (int)(w - item * B);
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    const int cv = colors[(int64_t)it.row * B + b];
    cnt[lane] = 0;
    __syncwarp();
    // pass 1: entries per color
    for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
      const int32_t e = e0 + lane;
      const int c = e < it.hi ? (int)colors[(int64_t)__ldg(col_idx + e) * B + b] : cv;
      const bool keep = c != cv;
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      const unsigned same = __match_any_sync(0xffffffffu, c) & km;
      if (keep && (same & lt) == 0) cnt[c] += __popc(same);
      __syncwarp();
    }
    // exclusive prefix over the colors (lane = color)
    const int x = cnt[lane];
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    cnt[lane] = incl - x;
    __syncwarp();
    // pass 2: place every kept entry after the earlier ones of its color
    int32_t* ids = gids + (int64_t)b * nnz + it.lo;
    uint8_t* cs = gcols + (int64_t)b * nnz + it.lo;
    for (int32_t e0 = it.lo; e0 < it.hi; e0 += 32) {
      const int32_t e = e0 + lane;
      const int32_t u = e < it.hi ? __ldg(col_idx + e) : 0;
      const int c = e < it.hi ? (int)colors[(int64_t)u * B + b] : cv;
      const bool keep = c != cv;
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      const unsigned same = __match_any_sync(0xffffffffu, c) & km;
      if (keep) {
        const int pos = cnt[c] + __popc(same & lt);
        ids[pos] = u;
        cs[pos] = (uint8_t)c;
      }
      __syncwarp();
      if (keep && (same & lt) == 0) cnt[c] += __popc(same);
      __syncwarp();
    }
    if (lane == 0) gkept[w] = total;
    __syncwarp();
  }
}

// Grouped form (one coloring per warp): a warp per (row or heavy-row segment,
// coloring b) walks the row's neighbours grouped by color (k_group_nbrs).
// Within a color group every neighbour's entry j lands at the same position
// of v's row, so the group's rows are summed in registers - lane l holds the
// entries j = j0 + l + 32 r (r < NR) of a chunk of 32 NR columns, read with
// coalesced loads - and each group's sum is added once into the output row in
// shared memory through the 16-bit position table [c_v][c_u][j] (0xFFFF =
// dropped).  Rows wider than a chunk walk the list once per chunk.  Summation
// order per position: CSR order within a color, colors ascending (fixed, so
// results are deterministic).
template <typename T, int B, int NR>
__global__ void __launch_bounds__(kBlock) k_spmm_g(
    const int32_t* __restrict__ row_ptr, int32_t n_seg, const int32_t* __restrict__ seg_row,
    const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi, int32_t n_heavy, int32_t n_act,
    const uint8_t* __restrict__ colors, int k, int64_t nnz, const int32_t* __restrict__ gids,
    const uint8_t* __restrict__ gcols, const int32_t* __restrict__ gkept, const T* __restrict__ Min, int w_in,
    int ld_in, T* __restrict__ P, int ld_out, T* __restrict__ scratch, const uint16_t* __restrict__ tab,
    const ScaleState* st_in, ScaleState* st_out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* acc = reinterpret_cast<T*>(sm_raw) + (int64_t)warp * ld_out;
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  float m = 0.f;
  for (int64_t w = blockIdx.x * (int64_t)wpb + warp; w < nitems * B; w += (int64_t)gridDim.x * wpb) {
    const int64_t item = w / B;
    const int b = (int)(w - item * B);
    const SpmmItem it = spmm_item(item, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    const int cv = colors[(int64_t)it.row * B + b];
    const int kept = gkept[w];
    for (int i = lane; i < ld_out; i += 32) acc[i] = T(0);
    __syncwarp();
    const int32_t* ids = gids + (int64_t)b * nnz + it.lo;
    const uint8_t* cs = gcols + (int64_t)b * nnz + it.lo;
    const uint16_t* tv = tab + (int64_t)cv * k * w_in;
    for (int j0 = 0; j0 < w_in; j0 += 32 * NR) {
      const int jl = j0 + lane;
      T a[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) a[r] = T(0);
      // a group's positions are distinct (one to one from a neighbour's columns), so all of a
      // lane's output words are read before any is written
      auto flush = [&](int c) {
        const uint16_t* tp = tv + (int64_t)c * w_in + jl;
        uint32_t pk[NR];
        T old[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) pk[r] = jl + 32 * r < w_in ? (uint32_t)__ldg(tp + 32 * r) : 0xFFFFu;
#pragma unroll
        for (int r = 0; r < NR; ++r) old[r] = pk[r] != 0xFFFFu ? acc[pk[r]] : T(0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (pk[r] != 0xFFFFu) acc[pk[r]] = old[r] + a[r];
          a[r] = T(0);
        }
        __syncwarp();
      };
      int cur = -1;
      // neighbour t's row entries are loaded while neighbour t - 1's are added (and a finished
      // group's sum is added into the output row), so two neighbours' loads are in flight (four,
      // measured, cost more registers than they hide latency)
      auto load = [&](int32_t u, T (&x)[NR]) {
        const T* src = Min + ((int64_t)u * ld_in + jl) * B + b;
#pragma unroll
        for (int r = 0; r < NR; ++r) x[r] = jl + 32 * r < w_in ? __ldg(src + 32 * r * B) : T(0);
      };
      for (int e0 = 0; e0 < kept; e0 += 32) {
        const int cnt = min(32, kept - e0);
        const int32_t u_lane = lane < cnt ? __ldg(ids + e0 + lane) : 0;
        const int c_lane = lane < cnt ? (int)__ldg(cs + e0 + lane) : 0;
        T x[NR];
        load(__shfl_sync(0xffffffffu, u_lane, 0), x);
        for (int t = 0; t < cnt; ++t) {
          const int c = __shfl_sync(0xffffffffu, c_lane, t);
          const int32_t un = __shfl_sync(0xffffffffu, u_lane, t + 1 < cnt ? t + 1 : t);
          T xn[NR];
          if (t + 1 < cnt) load(un, xn);
          if (c != cur) {
            if (cur >= 0) flush(cur);
            cur = c;
          }
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            a[r] += x[r];
            x[r] = xn[r];
          }
        }
      }
      if (cur >= 0) flush(cur);
    }
    T* dst = it.heavy ? scratch + item * (int64_t)ld_out * B : P + (int64_t)it.row * ld_out * B;
    for (int i = lane; i < ld_out; i += 32) {
      const T v = acc[i];
      dst[(int64_t)i * B + b] = v;
      if (!it.heavy) m = fmaxf(m, (float)v);
    }
    __syncwarp();
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
  }
}

// Staged grouped form (one coloring per pass, FP32): the sums of k_spmm_g, with
// the neighbour rows and the output positions copied into shared memory by
// 16-byte asynchronous copies (cp.async) instead of loaded into registers.  A
// warp's work is one sequence of entries: its items w0, w0 + S, ... (S warps in
// the grid), within an item the chunks of CH = 128 NR4 columns, within a chunk
// the kept neighbours in group order.  The copies run RS entries of it ahead
// of the entry being summed, across chunk and item boundaries: entry e's chunk
// of its neighbour's row goes to slot e % RS of a ring, and the first entry of
// a color group also copies the group's chunk of the position table (row pitch
// wp, a multiple of 8) into a ring of RS + 1 position buffers - the copies are
// at most RS groups ahead, so they never overwrite the group being summed.
// Every step commits one copy group (an empty one once the sequence is used
// up): the entry at the head has landed when all but the newest RS - 1 groups
// are done.  The entries' colors, known to every lane when they are issued,
// wait in a register queue of RS.  Lane l sums the columns j0 + 128 r + 4 l + q
// (r < NR4, q < 4).
// Per position the sums run in k_spmm_g's order (CSR order within a color,
// colors ascending): the same results.
template <int NR4, int RS>
__global__ void __launch_bounds__(512) k_spmm_gs(
    const int32_t* __restrict__ row_ptr, int32_t n_seg, const int32_t* __restrict__ seg_row,
    const int32_t* __restrict__ seg_lo, const int32_t* __restrict__ seg_hi, int32_t n_heavy, int32_t n_act,
    const uint8_t* __restrict__ colors, int k, const int32_t* __restrict__ gids, const uint8_t* __restrict__ gcols,
    const int32_t* __restrict__ gkept, const float* __restrict__ Min, int w_in, int ld_in, float* __restrict__ P,
    int ld_out, float* __restrict__ scratch, const uint16_t* __restrict__ tab, int wp, const ScaleState* st_in,
    ScaleState* st_out) {
  constexpr int CH = 128 * NR4;  // columns per chunk
  constexpr int PB = RS + 1;     // position buffers
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  // a warp's words: its output row, RS row chunks, PB chunks of 16-bit positions
  const int64_t per_warp = (int64_t)ld_out + RS * CH + PB * CH / 2;
  float* acc = reinterpret_cast<float*>(sm_raw) + warp * per_warp;
  float* slots = acc + ld_out;
  uint16_t* pbufs = reinterpret_cast<uint16_t*>(slots + RS * CH);
  const int64_t nitems = (int64_t)n_seg + (n_act - n_heavy);
  const int64_t S = (int64_t)gridDim.x * wpb;
  const int nch = (w_in + CH - 1) / CH;

  // the copies' cursor: item lw (lkept kept entries from llo on, row color lcv), chunk lc, entry
  // le; the ids and colors of the entries' block of 32 in lane registers; the last group's color
  int64_t lw = (int64_t)blockIdx.x * wpb + warp;
  int lc = 0, le = 0, lkept = 0, llo = 0, lcv = 0, lblk = -1, lprev = -1, lpb = 0;
  int32_t lid = 0;
  int lcol = 0;
  // the next item's kept count, first entry and row color, loaded when the copies enter an item
  // (independent loads, in flight while that item's rows are copied)
  int64_t nw = -1;
  int nk = 0, nlo = 0, ncv = 0;
  auto fetch = [&](int64_t w) {
    nw = w;
    if (w < nitems) {
      nk = gkept[w];
      const SpmmItem it = spmm_item(w, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
      nlo = it.lo;
      ncv = colors[it.row];
    }
  };
  auto seek = [&](int64_t w) -> int64_t {  // the first item from w on with kept entries
    for (; w < nitems; w += S) {
      int kk, lo = 0, cv = 0;
      if (w == nw) {
        kk = nk;
        lo = nlo;
        cv = ncv;
      } else {
        kk = gkept[w];
        if (kk > 0) {
          const SpmmItem it = spmm_item(w, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
          lo = it.lo;
          cv = colors[it.row];
        }
      }
      if (kk > 0) {
        lkept = kk;
        llo = lo;
        lcv = cv;
        lblk = -1;
        fetch(w + S);
        break;
      }
    }
    return w;
  };
  // copies the sequence's next entry into `slot` and returns its color (-1 past the end)
  auto issue = [&](int slot) -> int {
    int c = -1;
    if (lw < nitems) {
      const int blk = le >> 5;
      if (blk != lblk) {
        const int e = (blk << 5) + lane;
        lid = e < lkept ? __ldg(gids + llo + e) : 0;
        lcol = e < lkept ? (int)__ldg(gcols + llo + e) : 0;
        lblk = blk;
      }
      const int32_t u = __shfl_sync(full, lid, le & 31);
      c = __shfl_sync(full, lcol, le & 31);
      const int j0 = lc * CH;
      const int nv = (min(CH, w_in - j0) + 3) >> 2;  // 16-byte pieces of the row chunk
      const float* src = Min + (int64_t)u * ld_in + j0;
      float* dst = slots + slot * CH;
#pragma unroll
      for (int r = 0; r < NR4; ++r) {
        const int i = lane + 32 * r;
        if (i < nv) cp_async16(dst + 4 * i, src + 4 * i);
      }
      if (c != lprev) {  // a group starts: its chunk of positions
        const int np = min(CH, wp - j0) >> 3;  // 16-byte pieces of 8 positions
        const uint16_t* ps = tab + ((int64_t)lcv * k + c) * wp + j0;
        uint16_t* pd = pbufs + lpb * CH;
        for (int i = lane; i < np; i += 32) cp_async16(pd + 8 * i, ps + 8 * i);
        lpb = lpb + 1 == PB ? 0 : lpb + 1;
        lprev = c;
      }
      if (++le == lkept) {
        le = 0;
        lprev = -1;
        if (++lc == nch) {
          lc = 0;
          lw = seek(lw + S);
        }
      }
    }
    cp_async_commit();
    return c;
  };

  // the colors of the RS entries in flight, oldest first (every lane holds them)
  int cq[RS];
  lw = seek(lw);
#pragma unroll
  for (int i = 0; i < RS; ++i) cq[i] = issue(i);
  float m = 0.f;
  int slot = 0, cpb = 0;
  for (int64_t w = (int64_t)blockIdx.x * wpb + warp; w < nitems; w += S) {
    const SpmmItem it = spmm_item(w, n_seg, seg_row, seg_lo, seg_hi, n_heavy, row_ptr);
    const int kept = gkept[w];
    float4* acc4 = reinterpret_cast<float4*>(acc);
    for (int i = lane; i < ld_out / 4; i += 32) acc4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    for (int ch = 0; kept > 0 && ch < nch; ++ch) {
      const int j0 = ch * CH;
      float a[NR4][4];
#pragma unroll
      for (int r = 0; r < NR4; ++r) a[r][0] = a[r][1] = a[r][2] = a[r][3] = 0.f;
      int cur = -1;
      const uint16_t* pos = pbufs;
      // a group's positions are distinct (the map from a neighbour's columns to v's is one to
      // one), so a lane's output words are read before any is written: one shared-memory round
      // trip per 8 or 16 words instead of one per word (the positions and old values of all 4 NR4
      // words would not fit in registers beside the sums and the next chunk's words)
      auto flush = [&]() {
        constexpr int RB = NR4 == 8 ? 2 : NR4 < 4 ? NR4 : 4;  // 8 or 16 words at a time
#pragma unroll
        for (int r0 = 0; r0 < NR4; r0 += RB) {
          uint32_t pk[RB][4];
          float old[RB][4];
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            const int r = r0 + i, jb = j0 + 128 * r + 4 * lane;
            const uint2 pw = *reinterpret_cast<const uint2*>(pos + 128 * r + 4 * lane);
            pk[i][0] = jb < w_in ? pw.x & 0xffffu : 0xFFFFu;
            pk[i][1] = jb + 1 < w_in ? pw.x >> 16 : 0xFFFFu;
            pk[i][2] = jb + 2 < w_in ? pw.y & 0xffffu : 0xFFFFu;
            pk[i][3] = jb + 3 < w_in ? pw.y >> 16 : 0xFFFFu;
          }
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) old[i][q] = pk[i][q] != 0xFFFFu ? acc[pk[i][q]] : 0.f;
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (pk[i][q] != 0xFFFFu) acc[pk[i][q]] = old[i][q] + a[r0 + i][q];
              a[r0 + i][q] = 0.f;
            }
        }
        __syncwarp();
      };
      for (int e = 0; e < kept; ++e) {
        cp_async_wait<RS - 1>();
        __syncwarp();
        const int c = cq[0];
        // the entry's chunk is read before a group ends, so its loads overlap the flush
        const float4* s4 = reinterpret_cast<const float4*>(slots + slot * CH) + lane;
        float4 x[NR4];
#pragma unroll
        for (int r = 0; r < NR4; ++r) x[r] = s4[32 * r];
        if (c != cur) {
          if (cur >= 0) flush();
          cur = c;
          pos = pbufs + cpb * CH;
          cpb = cpb + 1 == PB ? 0 : cpb + 1;
        }
#pragma unroll
        for (int r = 0; r < NR4; ++r) {
          a[r][0] += x[r].x;
          a[r][1] += x[r].y;
          a[r][2] += x[r].z;
          a[r][3] += x[r].w;
        }
        __syncwarp();
        const int cn = issue(slot);
#pragma unroll
        for (int i = 0; i + 1 < RS; ++i) cq[i] = cq[i + 1];
        cq[RS - 1] = cn;
        slot = slot + 1 == RS ? 0 : slot + 1;
      }
      if (cur >= 0) flush();
    }
    float* dst = it.heavy ? scratch + w * (int64_t)ld_out : P + (int64_t)it.row * ld_out;
    float4* dst4 = reinterpret_cast<float4*>(dst);
    for (int i = lane; i < ld_out / 4; i += 32) {
      const float4 v = acc4[i];
      dst4[i] = v;
      if (!it.heavy) m = fmaxf(m, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  publish_max(st_out, m);
  if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_in->e;
}

// ------------------------------------------------------- general eMA --
// M_s(v, S) = sum over the splits (A, S \ A) of M_a(v, A) * P(v, S \ A).
// A block stages R consecutive rows of M_a and P in shared memory as
// [column][row] (row stride R+1), so that lanes - one row each, RPL rows per
// lane at stride 32 - read consecutive banks.  The split table holds the two
// shared-memory word offsets of every split (pre-multiplied by R+1); all
// lanes that share an output column read the same entry (a broadcast).
template <typename T, int R, int RPL>
__global__ void __launch_bounds__(kBlock) k_ema(
    const T* __restrict__ Ma, int64_t lda, int ca, const T* __restrict__ P, int64_t ldp, int cp,
    T* __restrict__ out, int64_t ldt, int ct, const uint2* __restrict__ tab, int nsplit, int sym, int64_t rows,
    int lb, const ScaleState* st_a, const ScaleState* st_p, ScaleState* st_out) {
  // element (row r, column c) of a table with row width ld: (r >> lb) * ld * batch + c * batch + (r & bmask)
  const int64_t bmask = (1 << lb) - 1;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  constexpr int RS = R + 1;
  constexpr int LPC = R >= 32 ? 32 : R;  // lanes sharing one output column
  constexpr int NSUB = 32 / LPC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int r = lane % LPC, sub = lane / LPC;
  // the symmetric form sums each unordered split once: the factor 2 is exact
  float scale = sym ? 2.f : 1.f;
  int s = 0;
  if (std::is_same<T, float>::value) {
    const float bound = (float)(sym ? 2 * nsplit : nsplit) * state_max(st_a) * state_max(st_p);
    s = shift_for(bound);
    scale *= pow2f(-s);
  }
  float m = 0.f;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < rows; r0 += (int64_t)gridDim.x * R) {
    const int nr = (int)(rows - r0 < R ? rows - r0 : R);
    __syncthreads();
    // staging: eight loads per thread in flight before their stores (wide rows stage
    // tens of KB per block, which a load-store-load loop would serialise on latency)
    auto stage = [&](const T* __restrict__ src, int64_t ld, int cols, int col0) {
      const int total = R * cols;
      for (int i0 = threadIdx.x; i0 < total; i0 += 8 * (int)blockDim.x) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * (int)blockDim.x;
          const int c = i / R, rr = i - c * R;
          const int64_t r = r0 + rr;
          v[u] = (i < total && rr < nr) ? src[(((r >> lb) * ld + c) << lb) + (r & bmask)] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * (int)blockDim.x;
          if (i < total) {
            const int c = i / R, rr = i - c * R;
            sm[(col0 + c) * RS + rr] = v[u];
          }
        }
      }
    };
    stage(Ma, lda, ca, 0);
    stage(P, ldp, cp, ca);
    __syncthreads();
    const T* base = sm + r;
    for (int S = warp * NSUB + sub; S < ldt; S += nwarp * NSUB) {
      T acc[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) acc[q] = T(0);
      if (S < ct) {
        const uint2* tp = tab + S;
        int j = 0;
        for (; j + 4 <= nsplit; j += 4) {
          const uint2 e0 = __ldg(tp), e1 = __ldg(tp + ct), e2 = __ldg(tp + 2 * ct), e3 = __ldg(tp + 3 * ct);
          tp += 4 * (int64_t)ct;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            acc[q] += base[e0.x + 32 * q] * base[e0.y + 32 * q];
            acc[q] += base[e1.x + 32 * q] * base[e1.y + 32 * q];
            acc[q] += base[e2.x + 32 * q] * base[e2.y + 32 * q];
            acc[q] += base[e3.x + 32 * q] * base[e3.y + 32 * q];
          }
        }
        for (; j < nsplit; ++j) {
          const uint2 e0 = __ldg(tp);
          tp += ct;
#pragma unroll
          for (int q = 0; q < RPL; ++q) acc[q] += base[e0.x + 32 * q] * base[e0.y + 32 * q];
        }
      }
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const T v = S < ct ? acc[q] * (T)scale : T(0);
        const int64_t rq = r0 + r + 32 * q;
        if (r + 32 * q < nr) out[(((rq >> lb) * ldt + S) << lb) + (rq & bmask)] = v;
        m = fmaxf(m, (float)v);
      }
    }
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_a->e + st_p->e + s;
  }
}

// ---- bulk copies (TMA, one-dimensional) into this CTA's shared memory, completed on an mbarrier --
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// wait for phase `parity` of the barrier, at most `limit` polls; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// eMA with a bank-conflict-free schedule (one coloring per pass).  A block
// stages R consecutive rows, each [M_a row | P row | 4 zero words] (the passive
// row starts `pofs` words in; a table combined with itself is staged once), by bulk
// copies completed on an mbarrier.  Outputs go in groups of 32, lane l of a
// group computing output 32 g + l for all R rows: the table orders each
// group's split terms in rounds in which the 32 lanes read 32 distinct banks
// of the active columns and 32 distinct banks of the passive ones (all lanes
// read the same row at a time), so each term costs two conflict-free shared
// loads for R multiply-adds, and a table word serves R rows.  Work units are
// (group, share of its rounds); with fewer groups than warps a group's rounds
// are split and the shares' partial sums added in share order, so results
// are deterministic.  A wait on the copies that runs out of polls writes NaN
// to the tile's outputs (which reaches the colorful maps) instead of hanging.
template <typename T, int R>
__global__ void __launch_bounds__(32 * kEmaSchedWarps) k_ema_s(
    const T* __restrict__ Ma, int64_t lda, const T* __restrict__ P, int64_t ldp, T* __restrict__ out, int64_t ldt,
    const uint32_t* __restrict__ tab, int G, int upg, int sym, int pofs, int rw, int64_t nv, int nsplit,
    const ScaleState* st_a, const ScaleState* st_p, ScaleState* st_out) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  T* rows = reinterpret_cast<T*>(sm_raw);
  T* part = rows + (int64_t)R * rw;                               // upg > 1: [unit][row][lane]
  uint64_t* bar = reinterpret_cast<uint64_t*>(part + (upg > 1 ? (int64_t)G * upg * 32 * R : 0));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float scale = sym ? 2.f : 1.f;
  int s = 0;
  if (std::is_same<T, float>::value) {
    const float bound = (float)(sym ? 2 * nsplit : nsplit) * state_max(st_a) * state_max(st_p);
    s = shift_for(bound);
    scale *= pow2f(-s);
  }
  if (threadIdx.x == 0) mbar_init(bar, 1);
  // every row ends in 4 zero words, which idle slots of the schedule read (no copy writes them)
  const int zofs = rw - 4;
  for (int i = threadIdx.x; i < 4 * R; i += blockDim.x) rows[(int64_t)(i >> 2) * rw + zofs + (i & 3)] = T(0);
  const uint32_t idle_e = (uint32_t)zofs | (uint32_t)(zofs - pofs) << 16;
  __syncthreads();
  const int nunits = G * upg;
  const uint32_t row_a = (uint32_t)(lda * (int64_t)sizeof(T)), row_p = (uint32_t)(ldp * (int64_t)sizeof(T));
  uint32_t parity = 0;
  float m = 0.f;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < nv; r0 += (int64_t)gridDim.x * R) {
    const int nr = (int)(nv - r0 < R ? nv - r0 : R);
    __syncthreads();  // every read of the previous tile is done
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(bar, (uint32_t)nr * (row_a + (sym ? 0u : row_p)));
      for (int r = 0; r < nr; ++r) {
        bulk_g2s(rows + (int64_t)r * rw, Ma + (r0 + r) * lda, row_a, bar);
        if (!sym) bulk_g2s(rows + (int64_t)r * rw + pofs, P + (r0 + r) * ldp, row_p, bar);
      }
    }
    const bool late = !mbar_wait(bar, parity, 1u << 24);
    parity ^= 1u;
    if (__syncthreads_or(late)) {  // the copies did not complete: poison this tile's outputs, all threads stop
      for (int64_t i = threadIdx.x; i < (int64_t)nr * ldt; i += blockDim.x)
        out[(r0 + i / ldt) * ldt + i % ldt] = T(NAN);
      return;
    }
    for (int u = warp; u < nunits; u += nwarps) {
      const int g = u / upg, share = u - g * upg;
      const uint32_t first = __ldg(tab + 2 * g), nrounds = __ldg(tab + 2 * g + 1);
      const uint32_t j0 = (uint32_t)(((uint64_t)nrounds * share) / upg);
      const uint32_t j1 = (uint32_t)(((uint64_t)nrounds * (share + 1)) / upg);
      const uint32_t* tp = tab + (int64_t)first * 32 + lane;
      T acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = T(0);
      // table words come eight rounds at a time, the next eight loaded while these are used (the
      // table streams from L2)
      uint32_t ev[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) ev[q] = j0 + q < j1 ? __ldg(tp + (int64_t)(j0 + q) * 32) : 0xFFFFFFFFu;
      for (uint32_t j = j0; j < j1; j += 8) {
        uint32_t en[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          en[q] = j + 8 + q < j1 ? __ldg(tp + (int64_t)(j + 8 + q) * 32) : 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t e = ev[q] == 0xFFFFFFFFu ? idle_e : ev[q];  // idle: the zero word (no branch)
          const T* pa = rows + (e & 0xFFFFu);
          const T* pp = rows + pofs + (e >> 16);
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r] += pa[(int64_t)r * rw] * pp[(int64_t)r * rw];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) ev[q] = en[q];
      }
      const int S = g * 32 + lane;
      if (upg == 1) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r < nr && S < ldt) {
            const T v = acc[r] * (T)scale;
            out[(r0 + r) * ldt + S] = v;
            m = fmaxf(m, (float)v);
          }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) part[((int64_t)u * R + r) * 32 + lane] = acc[r];
      }
    }
    if (upg > 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < G * 32 * R; i += blockDim.x) {
        const int g = i / (32 * R), r = (i / 32) % R, l = i % 32, S = g * 32 + l;
        if (r >= nr || S >= ldt) continue;
        T acc = T(0);
        for (int sh = 0; sh < upg; ++sh) acc += part[((int64_t)(g * upg + sh) * R + r) * 32 + l];
        const T v = acc * (T)scale;
        out[(r0 + r) * ldt + S] = v;
        m = fmaxf(m, (float)v);
      }
    }
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_a->e + st_p->e + s;
  }
}

// eMA for rows too wide to stage in shared memory (17 and 18 colors): one
// warp per row, lanes over the output columns, both operands read through L1
// at the raw split indices (I(A), I(S \ A)) of the table's [j][S] layout.
// Same sums, in the same order, as k_ema.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_ema_gl(
    const T* __restrict__ Ma, int64_t lda, const T* __restrict__ P, int64_t ldp, T* __restrict__ out, int64_t ldt,
    int ct, const uint2* __restrict__ tab, int nsplit, int sym, int64_t rows, int lb, const ScaleState* st_a,
    const ScaleState* st_p, ScaleState* st_out) {
  const int64_t bmask = (1 << lb) - 1;
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  float scale = sym ? 2.f : 1.f;
  int s = 0;
  if (std::is_same<T, float>::value) {
    const float bound = (float)(sym ? 2 * nsplit : nsplit) * state_max(st_a) * state_max(st_p);
    s = shift_for(bound);
    scale *= pow2f(-s);
  }
  float m = 0.f;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
    const T* a = Ma + (((r >> lb) * lda) << lb) + (r & bmask);
    const T* p = P + (((r >> lb) * ldp) << lb) + (r & bmask);
    T* o = out + (((r >> lb) * ldt) << lb) + (r & bmask);
    for (int S = lane; S < ldt; S += 32) {
      T acc = T(0);
      if (S < ct)
        for (int j = 0; j < nsplit; ++j) {
          const uint2 e = __ldg(tab + (int64_t)j * ct + S);
          acc += __ldg(a + ((int64_t)e.x << lb)) * __ldg(p + ((int64_t)e.y << lb));
        }
      const T v = S < ct ? acc * (T)scale : T(0);
      o[(int64_t)S << lb] = v;
      m = fmaxf(m, (float)v);
    }
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_a->e + st_p->e + s;
  }
}

// eMA over vertex tiles (batch B >= 4): a tile is V = (32 / B) * RPL
// vertices, whose whole interleaved rows (all B colorings, contiguous in the
// table) are copied into shared memory with 16-byte asynchronous copies -
// the next tile's while the current one is combined when two buffers fit
// (nbuf = 2).  The shared rows keep the global layout with a vertex stride
// vs == B (mod 32), so lane l = (vertex l / B, coloring l % B) reads a
// different bank for any column and a warp serves 32 rows of one output
// column S.  The table holds the raw split indices (I(A), I(S \ A)); the
// symmetric form (a table with itself) stages it once.  Same sums, in the
// same order, as k_ema.
template <typename T, int B, int RPL>
__global__ void __launch_bounds__(kBlock) k_ema_v(
    const T* __restrict__ Ma, int64_t lda, int ca, const T* __restrict__ P, int64_t ldp, int cp,
    T* __restrict__ out, int64_t ldt, int ct, const uint2* __restrict__ tab, int nsplit, int sym, int64_t nv, int vsa,
    int vsp, int nbuf, const ScaleState* st_a, const ScaleState* st_p, ScaleState* st_out) {
  constexpr int VPL = 32 / B;
  constexpr int V = VPL * RPL;
  constexpr int LB = B == 4 ? 2 : B == 8 ? 3 : B == 16 ? 4 : 5;
  constexpr int CH = 16 / (int)sizeof(T);  // elements per 16-byte copy
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int b = lane & (B - 1), vl0 = lane >> LB;
  const int buf_elems = V * vsa + (sym ? 0 : V * vsp);
  const int vs_p = sym ? vsa : vsp;
  float scale = sym ? 2.f : 1.f;
  int s = 0;
  if (std::is_same<T, float>::value) {
    const float bound = (float)(sym ? 2 * nsplit : nsplit) * state_max(st_a) * state_max(st_p);
    s = shift_for(bound);
    scale *= pow2f(-s);
  }
  const int64_t ntiles = (nv + V - 1) / V;
  const int na = (int)(lda * B / CH), np = (int)(ldp * B / CH);  // 16-byte chunks per vertex row
  auto issue = [&](int64_t tile, int bi) {
    T* dA = sm + (int64_t)bi * buf_elems;
    T* dP = dA + V * vsa;
    const int64_t v0 = tile * V;
    const int nvt = (int)(nv - v0 < V ? nv - v0 : V);
    for (int i = threadIdx.x; i < nvt * na; i += blockDim.x) {
      const int vl = i / na, c = i - vl * na;
      cp_async16(dA + vl * vsa + c * CH, Ma + ((v0 + vl) * lda * B + (int64_t)c * CH));
    }
    if (!sym)
      for (int i = threadIdx.x; i < nvt * np; i += blockDim.x) {
        const int vl = i / np, c = i - vl * np;
        cp_async16(dP + vl * vsp + c * CH, P + ((v0 + vl) * ldp * B + (int64_t)c * CH));
      }
  };
  float m = 0.f;
  int bi = 0;
  int64_t tile = blockIdx.x;
  if (tile < ntiles) issue(tile, 0);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t next = tile + gridDim.x;
    if (nbuf == 2) {
      if (next < ntiles) issue(next, bi ^ 1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* A = sm + (int64_t)bi * buf_elems;
    const T* Pp = sym ? A : A + V * vsa;
    const int64_t v0 = tile * V;
    for (int S = warp; S < ldt; S += nwarp) {
      T acc[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) acc[q] = T(0);
      if (S < ct) {
        const uint2* tp = tab + S;
        int j = 0;
        for (; j + 2 <= nsplit; j += 2) {
          const uint2 e0 = __ldg(tp), e1 = __ldg(tp + ct);
          tp += 2 * (int64_t)ct;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int va = (vl0 + VPL * q) * vsa + b, vp = (vl0 + VPL * q) * vs_p + b;
            acc[q] += A[va + (int)(e0.x << LB)] * Pp[vp + (int)(e0.y << LB)];
            acc[q] += A[va + (int)(e1.x << LB)] * Pp[vp + (int)(e1.y << LB)];
          }
        }
        if (j < nsplit) {
          const uint2 e0 = __ldg(tp);
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int va = (vl0 + VPL * q) * vsa + b, vp = (vl0 + VPL * q) * vs_p + b;
            acc[q] += A[va + (int)(e0.x << LB)] * Pp[vp + (int)(e0.y << LB)];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int64_t v = v0 + vl0 + VPL * q;
        const T val = S < ct ? acc[q] * (T)scale : T(0);
        if (v < nv) {
          out[(v * ldt + S) * B + b] = val;
          m = fmaxf(m, (float)val);
        }
      }
    }
    __syncthreads();  // every warp is done with this buffer before it is refilled
    if (nbuf == 2) {
      bi ^= 1;
    } else {
      if (next < ntiles) issue(next, 0);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_a->e + st_p->e + s;
  }
}

// eMA with every operand in registers, for a few (K, a-1, p) shapes compiled
// in: one thread per (vertex, coloring) row holds the passive row P(v, .)
// and the output row in registers and streams the active row: for each
// (a-1)-subset A of the K relative colors, M_a(v, A) is loaded (or, in the
// symmetric form, taken from the registers) once and multiplied into every
// output S = A + S_p over the p-subsets S_p of the other colors.  The splits
// are fixed by the subset sizes alone (both rows are relative to the same
// color c(v)), so their index pairs are constants generated at compile time
// and the FMAs address registers directly: no table, no shared memory, and
// the kernel streams the three tables once (HBM-bound instead of bound by
// shared-memory operand reads).  The A subsets are visited in decreasing
// mask order, the order in which the split table lists the splits of every
// S, so each output receives its terms in the same order as k_ema / k_ema_v:
// the FP32 sums are the same.
__host__ __device__ constexpr int c_binom(int n, int r) {
  if (r < 0 || r > n) return 0;
  int64_t x = 1;
  for (int i = 1; i <= r; ++i) x = x * (n - r + i) / i;
  return (int)x;
}
__host__ __device__ constexpr int c_popc(uint32_t m) {
  int c = 0;
  for (; m; m >>= 1) c += (int)(m & 1u);
  return c;
}
// Eq. 1: colex rank of the set of ascending colors c_1 < c_2 < ..: sum_i C(c_i, i)
__host__ __device__ constexpr int c_rank(uint32_t m) {
  int r = 0, i = 0;
  for (int c = 0; c < 32; ++c)
    if (m >> c & 1u) r += c_binom(c, ++i);
  return r;
}

template <int K, int AR, int PR, bool SYM>
struct EmaRegPlan {
  static constexpr int NA = c_binom(K, AR), NP = c_binom(K, PR), NO = c_binom(K, AR + PR);
  static constexpr int NPAIR = NO * (SYM ? c_binom(AR + PR, AR) / 2 : c_binom(AR + PR, AR));
  struct Tab {
    int16_t ga[NA];         // A index of group g (groups in decreasing mask order)
    int16_t g0[NA + 1];     // first pair of group g
    int16_t p[NPAIR], o[NPAIR];
  };
  static constexpr Tab make() {
    Tab t{};
    int n = 0, g = 0;
    for (uint32_t m = 1u << K; m-- > 0;) {
      if (c_popc(m) != AR) continue;
      const uint32_t rest = ((1u << K) - 1) & ~m;
      t.ga[g] = (int16_t)c_rank(m);
      t.g0[g] = (int16_t)n;
      for (uint32_t s = rest;; s = (s - 1) & rest) {
        if (c_popc(s) == PR && (!SYM || c_rank(m) < c_rank(s))) {
          t.p[n] = (int16_t)c_rank(s);
          t.o[n] = (int16_t)c_rank(m | s);
          ++n;
        }
        if (s == 0) break;
      }
      ++g;
    }
    t.g0[g] = (int16_t)n;
    return t;
  }
  static constexpr Tab tab = make();
  __host__ __device__ static constexpr int ga(int g) { return tab.ga[g]; }
  __host__ __device__ static constexpr int g0(int g) { return tab.g0[g]; }
  __host__ __device__ static constexpr int gn(int g) { return tab.g0[g + 1] - tab.g0[g]; }
  __host__ __device__ static constexpr int pi(int i) { return tab.p[i]; }
  __host__ __device__ static constexpr int oi(int i) { return tab.o[i]; }
};
template <int V>
struct CInt {
  static constexpr int v = V;
};

template <class PL, int G, int... J>
__device__ __forceinline__ void ema_reg_group(float a, const float (&p)[PL::NP], float (&o)[PL::NO],
                                              std::integer_sequence<int, J...>) {
  ((o[CInt<PL::oi(PL::g0(G) + J)>::v] =
        fmaf(a, p[CInt<PL::pi(PL::g0(G) + J)>::v], o[CInt<PL::oi(PL::g0(G) + J)>::v])),
   ...);
}
template <class PL, bool SYM, int... G>
__device__ __forceinline__ void ema_reg_groups(const float* __restrict__ A, int B, const float (&p)[PL::NP],
                                               float (&o)[PL::NO], std::integer_sequence<int, G...>) {
  (ema_reg_group<PL, G>(SYM ? p[CInt<PL::ga(G)>::v] : __ldg(A + PL::ga(G) * B), p, o,
                        std::make_integer_sequence<int, PL::gn(G)>{}),
   ...);
}
template <int... I>
__device__ __forceinline__ void ema_reg_load(const float* __restrict__ src, int B, float* p,
                                             std::integer_sequence<int, I...>) {
  ((p[I] = __ldg(src + I * B)), ...);
}

template <int K, int AR, int PR, bool SYM>
__global__ void __launch_bounds__(128, SYM ? 3 : 2) k_ema_reg(const float* __restrict__ Ma, int64_t lda,
                                                 const float* __restrict__ P, int64_t ldp, float* __restrict__ out,
                                                 int64_t ldt, int64_t nv, int lb, const ScaleState* st_a,
                                                 const ScaleState* st_p, ScaleState* st_out) {
  using PL = EmaRegPlan<K, AR, PR, SYM>;
  const int B = 1 << lb;
  const int nsplit = SYM ? c_binom(AR + PR, AR) / 2 : c_binom(AR + PR, AR);
  const float bound = (float)(SYM ? 2 * nsplit : nsplit) * state_max(st_a) * state_max(st_p);
  const int s = shift_for(bound);
  const float scale = (SYM ? 2.f : 1.f) * pow2f(-s);
  const int64_t rows = nv << lb;
  float m = 0.f;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = r >> lb;
    const int b = (int)(r & (B - 1));
    float p[PL::NP], o[PL::NO];
    ema_reg_load(P + v * ldp * B + b, B, p, std::make_integer_sequence<int, PL::NP>{});
#pragma unroll
    for (int i = 0; i < PL::NO; ++i) o[i] = 0.f;
    ema_reg_groups<PL, SYM>(Ma + v * lda * B + b, B, p, o, std::make_integer_sequence<int, PL::NA>{});
    float* dst = out + v * ldt * B + b;
#pragma unroll
    for (int i = 0; i < PL::NO; ++i) {
      const float x = o[i] * scale;
      dst[(int64_t)i * B] = x;
      m = fmaxf(m, x);
    }
    for (int64_t i = PL::NO; i < ldt; ++i) dst[i * B] = 0.f;
  }
  publish_max(st_out, m);
  if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = st_a->e + st_p->e + s;
}

// the (K, a-1, p, symmetric) shapes compiled in: the 10-color spider's combine
// of a 3-vertex leg with the root and another leg (and its symmetric form), and
// the combines the 7-, 8- and 11-vertex Pruefer trees (seeds 1007, 1008, 1011)
// plan at 8 or more colorings per pass, whose passive and output rows fit in
// registers (C(K, p) + C(K, a-1+p) at most 165 floats)
#define SGC_EMA_REG_SHAPES(X) \
  X(9, 3, 3, false)           \
  X(9, 3, 3, true)            \
  X(6, 3, 2, false)           \
  X(7, 1, 1, true)            \
  X(10, 2, 1, false)          \
  X(10, 1, 1, true)           \
  X(10, 5, 3, false)

// ----------------------------------------------- last step + vertex sum --
// maps_b = sum_v sum_{C_p} M_a(v, [k] \ C_p) * P(v, C_p).  One thread per row
// r = v * batch + b, rows r, r + S, ... with S (the grid's thread count) a
// multiple of the batch, so a thread always serves the same coloring.  A row's
// products are summed in the table type (exact for FP64 integers; in FP32
// the products of values <= 1 and <= max degree cannot overflow) and the
// per-vertex totals in FP64; per-block partials per coloring are summed in
// block order by k_final_sum, so the result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_final(const T* __restrict__ Ma, int64_t lda, const T* __restrict__ P,
                                                  int64_t ldp, int cp, const uint32_t* __restrict__ tab,
                                                  int64_t rows, int lb, double* __restrict__ partials) {
  __shared__ double tacc[kBlock];
  const int batch = 1 << lb;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += S) {
    const int64_t v = row >> lb, b = row & (batch - 1);
    const T* a = Ma + (v * lda << lb) + b;
    const T* pp = P + (v * ldp << lb) + b;
    T part = T(0);
    for (int i = 0; i < cp; ++i) {
      const uint32_t ia = __ldg(tab + i);
      if (ia < (uint32_t)lda) part += a[(int64_t)ia << lb] * pp[(int64_t)i << lb];
    }
    acc += (double)part;
  }
  tacc[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < batch) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += batch) s += tacc[i];
    partials[(int64_t)blockIdx.x * batch + threadIdx.x] = s;
  }
}

// k_final for a (K, p) compiled in (SGC_FINAL_REG_SHAPES): the active index of
// each passive color set - the rank of its complement among the K relative
// colors - is a compile-time constant, so the loop over the C(K, p) sets is
// fully unrolled with no table loads and the loads of a row are all
// independent (many in flight per thread).  Same rows per thread, same
// per-row order and same per-block sums as k_final: the same results.
template <int K, int PR>
struct FinalRegPlan {
  static constexpr int NP = c_binom(K, PR);
  struct Tab {
    int16_t ia[NP];
  };
  static constexpr Tab make() {
    Tab t{};
    const uint32_t full = (1u << K) - 1;
    for (uint32_t m = 0; m <= full; ++m)
      if (c_popc(m) == PR) t.ia[c_rank(m)] = (int16_t)c_rank(full & ~m);
    return t;
  }
  static constexpr Tab tab = make();
  __host__ __device__ static constexpr int ia(int i) { return tab.ia[i]; }
};
template <typename T, class FP, int... I>
__device__ __forceinline__ T final_reg_row(const T* __restrict__ a, const T* __restrict__ p, int lb,
                                           std::integer_sequence<int, I...>) {
  const T av[] = {__ldg(a + ((int64_t)CInt<FP::ia(I)>::v << lb))...};
  const T pv[] = {__ldg(p + ((int64_t)I << lb))...};
  T part = T(0);
  ((part += av[I] * pv[I]), ...);
  return part;
}
template <typename T, int K, int PR>
__global__ void __launch_bounds__(kBlock, 2) k_final_reg(const T* __restrict__ Ma, int64_t lda,
                                                         const T* __restrict__ P, int64_t ldp, int64_t rows, int lb,
                                                         double* __restrict__ partials) {
  using FP = FinalRegPlan<K, PR>;
  __shared__ double tacc[kBlock];
  const int batch = 1 << lb;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += S) {
    const int64_t v = row >> lb, b = row & (batch - 1);
    acc += (double)final_reg_row<T, FP>(Ma + (v * lda << lb) + b, P + (v * ldp << lb) + b, lb,
                                        std::make_integer_sequence<int, FP::NP>{});
  }
  tacc[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < batch) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += batch) s += tacc[i];
    partials[(int64_t)blockIdx.x * batch + threadIdx.x] = s;
  }
}

// the (K, p) shapes of the last step compiled in: the 10-color spider's, the 7-, 8-, 9- and
// 11-vertex Pruefer trees' and the 15-vertex one's (the 10-vertex tree's (9, 5), 126 terms per
// row, spills registers and keeps the table form)
#define SGC_FINAL_REG_SHAPES(X) \
  X(9, 3) X(6, 1) X(7, 3) X(8, 4) X(10, 2) X(14, 1) X(14, 13)

// The symmetric register-form eMA fused with the last step that consumes it:
// the root's table T(v, .) = sum over splits of P(v, A) P(v, S - A) (as in
// k_ema_reg, in registers, scaled the same way) is never stored; each row's
// last-step term sum over the p-sets C of T(v, complement of C) P(v, C) is
// taken from the registers in k_final_reg's order, and the rows' sums go into
// per-block FP64 partials for k_final_sum.  Rows r = v B + b, r + S, ... with S
// the grid's thread count (a multiple of B), so a thread keeps one coloring.
template <class FP, int N, int... I>
__device__ __forceinline__ float ema_final_row(const float (&o)[N], const float (&p)[N], std::integer_sequence<int, I...>) {
  float part = 0.f;
  ((part += o[CInt<FP::ia(I)>::v] * p[I]), ...);
  return part;
}
template <int K, int PR>
__global__ void __launch_bounds__(128, 3) k_ema_final_reg(const float* __restrict__ P, int64_t ldp, int64_t rows,
                                                          int lb, const ScaleState* st_p, ScaleState* st_t,
                                                          double* __restrict__ partials) {
  using PL = EmaRegPlan<K, PR, PR, true>;
  using FP = FinalRegPlan<K, PR>;
  static_assert(PL::NO == FP::NP, "the root table's width is the passive table's");
  __shared__ double tacc[128];
  const int B = 1 << lb;
  const int nsplit = c_binom(2 * PR, PR) / 2;
  const float bound = (float)(2 * nsplit) * state_max(st_p) * state_max(st_p);
  const int s = shift_for(bound);
  const float scale = 2.f * pow2f(-s);
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += S) {
    const int64_t v = r >> lb;
    const int b = (int)(r & (B - 1));
    const float* src = P + v * ldp * B + b;
    float p[PL::NP], o[PL::NO];
    ema_reg_load(src, B, p, std::make_integer_sequence<int, PL::NP>{});
#pragma unroll
    for (int i = 0; i < PL::NO; ++i) o[i] = 0.f;
    ema_reg_groups<PL, true>(src, B, p, o, std::make_integer_sequence<int, PL::NA>{});
#pragma unroll
    for (int i = 0; i < PL::NO; ++i) o[i] *= scale;
    acc += (double)ema_final_row<FP>(o, p, std::make_integer_sequence<int, FP::NP>{});
  }
  tacc[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < B) {
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += B) t += tacc[i];
    partials[(int64_t)blockIdx.x * B + threadIdx.x] = t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st_t->e = 2 * st_p->e + s;
}

// the (K, p) shapes of the fused combine + last step compiled in: the 10-color spider's
#define SGC_EMA_FINAL_SHAPES(X) X(9, 3)


// last step with a single-vertex active child: maps_b = sum_v P(v, all colors but c(v)),
// the single entry of the relative P row
template <typename T>
__global__ void __launch_bounds__(kBlock) k_final_leaf(const T* __restrict__ P, int64_t ldp, int64_t rows, int lb,
                                                       double* __restrict__ partials) {
  __shared__ double tacc[kBlock];
  const int batch = 1 << lb;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;  // multiple of batch
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += S)
    acc += (double)P[((row >> lb) * ldp << lb) + (row & (batch - 1))];
  tacc[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < batch) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += batch) s += tacc[i];
    partials[(int64_t)blockIdx.x * batch + threadIdx.x] = s;
  }
}

// Ablation of the pruning (Eq. 2, Section 4.2): one combine in Algorithm 1's
// loop order - for every row, output color set and split the neighbour sum is
// taken again, instead of once per passive color set (no SpMM).  One thread
// per (row, output color set).  A single-vertex child's table is all ones and
// not stored (Ma / Mp null).  npos[c_v][I_p][c_u] is the index of the split's
// p-set minus c_u in a neighbour's passive row (~0: the neighbour adds nothing).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_unpruned(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n_act,
    const uint8_t* __restrict__ colors, int lb, int k, const T* __restrict__ Ma, int64_t lda,
    const T* __restrict__ Mp, int64_t ldp, int wp, T* __restrict__ out, int64_t ldt, int ct,
    const uint2* __restrict__ tab, int nsplit, const uint32_t* __restrict__ npos, int max_deg,
    const ScaleState* st_a, const ScaleState* st_p, ScaleState* st_out) {
  const int batch = 1 << lb;
  float scale = 1.f;
  int s = 0;
  if (std::is_same<T, float>::value) {
    const float ma = st_a ? state_max(st_a) : 1.f, mp = st_p ? state_max(st_p) : 1.f;
    s = shift_for((float)nsplit * (float)max_deg * ma * mp);
    scale = pow2f(-s);
  }
  float m = 0.f;
  const int64_t items = ((int64_t)n_act << lb) * ldt;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = it / ldt;
    const int S = (int)(it - r * ldt);
    const int64_t v = r >> lb;
    const int b = (int)(r & (batch - 1));
    T acc = T(0);
    if (S < ct) {
      const int cv = colors[v * batch + b];
      const uint32_t* np0 = npos + (int64_t)cv * wp * k;
      for (int j = 0; j < nsplit; ++j) {
        const uint2 e = __ldg(tab + (int64_t)j * ct + S);
        const T a = Ma ? Ma[((v * lda + e.x) << lb) + b] : T(1);
        if (a == T(0)) continue;
        const uint32_t* np = np0 + (int64_t)e.y * k;
        T sum = T(0);
        for (int32_t q = row_ptr[v]; q < row_ptr[v + 1]; ++q) {
          const int32_t u = __ldg(col_idx + q);
          const uint32_t pj = __ldg(np + colors[(int64_t)u * batch + b]);
          if (pj != 0xFFFFFFFFu) sum += Mp ? Mp[(((int64_t)u * ldp + pj) << lb) + b] : T(1);
        }
        acc += a * sum;
      }
    }
    const T val = acc * (T)scale;
    out[((v * ldt + S) << lb) + b] = val;
    m = fmaxf(m, (float)val);
  }
  if (std::is_same<T, float>::value) {
    publish_max(st_out, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) st_out->e = (st_a ? st_a->e : 0) + (st_p ? st_p->e : 0) + s;
  }
}

// More colors than template vertices (Section 2.1, k >= |T|): maps_b = sum_v of
// all entries of the root table row (every |T|-subset of colors containing
// c(v)); summed like k_final: the row in the table type, vertices in FP64,
// per-block partials per coloring.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_final_rows(const T* __restrict__ M, int64_t ld, int cols, int64_t rows,
                                                       int lb, double* __restrict__ partials) {
  __shared__ double tacc[kBlock];
  const int batch = 1 << lb;
  const int64_t S = (int64_t)gridDim.x * blockDim.x;  // multiple of batch
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += S) {
    const T* m = M + (((row >> lb) * ld) << lb) + (row & (batch - 1));
    T part = T(0);
    for (int i = 0; i < cols; ++i) part += m[(int64_t)i << lb];
    acc += (double)part;
  }
  tacc[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < batch) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)blockDim.x; i += batch) s += tacc[i];
    partials[(int64_t)blockIdx.x * batch + threadIdx.x] = s;
  }
}

__global__ void k_final_sum(const double* __restrict__ partials, int nblocks, int batch, const ScaleState* st_a,
                            const ScaleState* st_p, int fp32, double* __restrict__ out) {
  const int b = threadIdx.x;
  if (b >= batch) return;
  double s = 0.0;
  for (int i = 0; i < nblocks; ++i) s += partials[(int64_t)i * batch + b];
  if (fp32) {
    const int e = (st_a ? st_a->e : 0) + st_p->e;
    s = ldexp(s, e);
  }
  out[b] = s;
}

// A kernel's limit on dynamic shared memory only ever grows, per device: one kernel serves ops of
// different sizes, and a launch recorded into a CUDA graph with a larger size must not find the
// limit lowered by a later, smaller launch (a profiler that replays graph nodes one by one
// checks each node against the kernel's limit at that time).
std::mutex g_smem_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_limit;

template <typename KernelT>
void allow_smem(KernelT kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_smem_mu);
  size_t& cur = g_smem_limit[{dev, reinterpret_cast<const void*>(kernel)}];
  if (bytes <= cur) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    cur = bytes;
}

int grid_for(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <typename T, bool BUCKETS, int NSMAX, int PT = 0>
void launch_spmm_k(const sgc_graph* g, const PlanOp& op, int batch, int k, const uint8_t* colors, const T* M, T* P,
                   T* scratch, const uint32_t* tab, int tab_smem, const ScaleState* si, ScaleState* so, int wpb,
                   size_t smem, cudaStream_t st, int tab_ld = 0, int grid_cap = 1 << 30) {
  allow_smem(k_spmm<T, BUCKETS, NSMAX, PT>, smem);
  const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
  k_spmm<T, BUCKETS, NSMAX, PT><<<grid_for(nitems, wpb, grid_cap), 32 * wpb, smem, st>>>(
      g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, colors,
      batch, k, op.p, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.cols_out, (int)op.ld_out, scratch, tab, tab_smem,
      tab_ld > 0 ? tab_ld : (int)op.cols_p, si, so);
}

// Launch shape of the SpMM: the direct form keeps a plain loop (few registers,
// high occupancy); the bucketed form (small buckets) uses the pipelined loop.
template <typename T>
sgc_status launch_spmm(const sgc_graph* g, const PlanOp& op, int batch, int k, const uint8_t* colors, const T* M,
                       T* P, T* scratch, const uint32_t* tab, const ScaleState* si, ScaleState* so, int num_sms,
                       size_t smem_cap, cudaStream_t st, int64_t* nk) {
  if (op.spmm_buckets && op.spmm_variant == 2) {
    // register buckets: one coloring per pass; wpr warps of 32 * NS columns per row
    if (batch != 1) return fail(SGC_ERR_INTERNAL, "register-bucket SpMM needs one coloring per pass");
    const int w_in = (int)op.cols_p;
    const int ns = w_in <= 32 ? 1 : w_in <= 512 ? 2 : 4;
    const int wpr = (w_in + 32 * ns - 1) / (32 * ns);
    if (wpr > kBlock / 32 || k > 16) return fail(SGC_ERR_UNSUPPORTED, "SpMM row too wide for register buckets");
    const int rows = (kBlock / 32) / wpr;
    const size_t smem_rb = (size_t)rows * k * w_in * sizeof(T);
    if (smem_rb > smem_cap) return fail(SGC_ERR_UNSUPPORTED, "register-bucket rows do not fit in shared memory");
    const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
    const int threads = rows * wpr * 32;
#define SGC_RB(NS_)                                                                                          \
  do {                                                                                                       \
    allow_smem(k_spmm_rb<T, NS_>, smem_rb);                                                                  \
    k_spmm_rb<T, NS_><<<grid_for(nitems, rows, 1 << 30), threads, smem_rb, st>>>(                           \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, \
        colors, k, op.p, M, w_in, (int)op.ld_p, P, (int)op.cols_out, (int)op.ld_out, scratch, tab, wpr, si,   \
        so);                                                                                                 \
  } while (0)
    if (ns == 1) SGC_RB(1);
    else if (ns == 2) SGC_RB(2);
    else SGC_RB(4);
#undef SGC_RB
    ++*nk;
    if (g->n_heavy > 0) {
      constexpr int VN = Vec16<T>::n;
      k_spmm_reduce<T><<<grid_for((int64_t)g->n_heavy * (op.ld_out / VN), kBlock, 16 * num_sms), kBlock, 0, st>>>(
          g->d_heavy_seg, g->n_heavy, scratch, op.ld_out, P, op.ld_out, so);
      ++*nk;
    }
    return SGC_OK;
  }
  const size_t per_warp = op.spmm_buckets ? (size_t)spmm_bucket_bytes(batch, k, op.cols_p, (int)sizeof(T))
                                          : (size_t)batch * op.ld_out * sizeof(T);
  // the bucketed form's resolve table is staged in shared memory when small;
  // the direct form reads its position table through L1 (staging it in shared
  // memory measured slower: bank conflicts on the scattered lookups)
  const int64_t tab_words = (int64_t)k * op.cols_out * op.p;
  const int pos_bytes = op.spmm_buckets ? 0 : op.spmm_pos_bytes;
  const int64_t packed_ld = pos_bytes ? spmm_packed_ld(op.cols_p, pos_bytes) : 0;
  const int tab_smem = pos_bytes ? (int)(((int64_t)k * k * packed_ld * pos_bytes + 3) / 4)
                       : op.spmm_buckets && tab_words * 4 <= 16 * 1024 ? (int)tab_words
                                                                        : 0;
  int wpb = kBlock / 32;
  while (wpb > 1 && per_warp * wpb + (size_t)tab_smem * 4 > smem_cap) wpb /= 2;
  if (per_warp * wpb + (size_t)tab_smem * 4 > smem_cap)
    return fail(SGC_ERR_UNSUPPORTED, "SpMM row does not fit in shared memory");
  const size_t smem = per_warp * wpb + (size_t)tab_smem * 4;
  if (op.spmm_buckets && op.spmm_variant == 7) {
    const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
#define SGC_BK(B_)                                                                                           \
  do {                                                                                                       \
    allow_smem(k_spmm_bk<T, B_>, smem);                                                                      \
    k_spmm_bk<T, B_><<<grid_for(nitems, wpb, 1 << 30), 32 * wpb, smem, st>>>(                               \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, \
        colors, k, op.p, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.cols_out, (int)op.ld_out, scratch, tab, \
        tab_smem, si, so);                                                                                   \
  } while (0)
    switch (batch) {
      case 1: SGC_BK(1); break;
      case 2: SGC_BK(2); break;
      case 4: SGC_BK(4); break;
      case 8: SGC_BK(8); break;
      case 16: SGC_BK(16); break;
      default: SGC_BK(32); break;
    }
#undef SGC_BK
  } else if (op.spmm_buckets) {
    const int64_t per_lane = (op.cols_p + 32 / batch - 1) / (32 / batch);
    if (per_lane <= 4)
      launch_spmm_k<T, true, 4>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st);
    else if (per_lane <= 8)
      launch_spmm_k<T, true, 8>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st);
    else if (per_lane <= 16)
      launch_spmm_k<T, true, 16>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st);
    else
      launch_spmm_k<T, true, 0>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st);
  } else {
    const int64_t per_lane = (op.cols_p + 32 / batch - 1) / (32 / batch);
    const int variant = op.spmm_variant;
    const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
#define SGC_DIRECT_PF(NS_)                                                                                      \
  do {                                                                                                          \
    allow_smem(k_spmm_direct_pf<T, NS_>, smem);                                                                 \
    k_spmm_direct_pf<T, NS_><<<grid_for(nitems, wpb, 1 << 30), 32 * wpb, smem, st>>>(                         \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act,     \
        colors, batch, k, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.ld_out, scratch, tab, si, so);           \
  } while (0)
    if (variant == 12) {
      const uint4* tab4 = reinterpret_cast<const uint4*>(tab);
      if (op.ld_out >= 65535) return fail(SGC_ERR_UNSUPPORTED, "wide SpMM: positions must fit 16 bits");
#define SGC_W(B_)                                                                                              \
  do {                                                                                                         \
    allow_smem(k_spmm_w<T, B_>, smem);                                                                         \
    k_spmm_w<T, B_><<<grid_for(nitems, wpb, 1 << 30), 32 * wpb, smem, st>>>(                                   \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act,   \
        colors, k, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.ld_out, scratch, tab4, si, so);                \
  } while (0)
      switch (batch) {
        case 1: SGC_W(1); break;
        case 2: SGC_W(2); break;
        case 4: SGC_W(4); break;
        case 8: SGC_W(8); break;
        case 16: SGC_W(16); break;
        default: SGC_W(32); break;
      }
#undef SGC_W
    } else if (variant == 11) {
      const int L = 32 / batch;
      const int64_t nsmax = (op.cols_p + L - 1) / L;
      const uint4* tab4 = reinterpret_cast<const uint4*>(tab);
#define SGC_U(B_, NS_)                                                                                         \
  do {                                                                                                         \
    allow_smem(k_spmm_u<T, B_, NS_>, smem);                                                                    \
    k_spmm_u<T, B_, NS_><<<grid_for(nitems, wpb, 1 << 30), 32 * wpb, smem, st>>>(                              \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act,   \
        colors, k, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.ld_out, scratch, tab4, si, so);                \
  } while (0)
#define SGC_U2(B_)                 \
  do {                             \
    if (nsmax <= 3)                \
      SGC_U(B_, 3);                \
    else if (nsmax <= 4)           \
      SGC_U(B_, 4);                \
    else if (nsmax <= 8)           \
      SGC_U(B_, 8);                \
    else if (nsmax <= 9)           \
      SGC_U(B_, 9);                \
    else if (nsmax <= 12)          \
      SGC_U(B_, 12);               \
    else                           \
      SGC_U(B_, 16);               \
  } while (0)
      if (nsmax > 16 || op.ld_out > 255 || (batch != 4 && batch != 8 && batch != 16))
        return fail(SGC_ERR_UNSUPPORTED, "unrolled SpMM: needs 4..16 colorings, <= 16 entries per lane, < 255 positions");
      if (batch == 4) SGC_U2(4);
      else if (batch == 8) SGC_U2(8);
      else SGC_U2(16);
#undef SGC_U2
#undef SGC_U
    } else if (variant == 5 || variant == 6 || variant == 8 || variant == 9 || variant == 10) {
#define SGC_D(B_, LM_, G_)                                                                                   \
  do {                                                                                                       \
    allow_smem(k_spmm_d<T, B_, LM_, G_>, smem);                                                              \
    k_spmm_d<T, B_, LM_, G_><<<grid_for(nitems, wpb, 1 << 30), 32 * wpb, smem, st>>>(                       \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, \
        colors, k, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.ld_out, scratch, tab, nsp, si, so);         \
  } while (0)
#define SGC_DP(B_)                                                                                           \
  do {                                                                                                       \
    allow_smem(k_spmm_d<T, B_, false, 0, true>, smem_priv);                                                  \
    k_spmm_d<T, B_, false, 0, true><<<grid_for(nitems, wpb_priv, 1 << 30), 32 * wpb_priv, smem_priv, st>>>( \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, \
        colors, k, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.ld_out, scratch, tab, nsp, si, so);         \
  } while (0)
#define SGC_D2(B_)                   \
  do {                               \
    if (variant == 10)               \
      SGC_DP(B_);                    \
    else if (variant == 6)           \
      SGC_D(B_, true, 0);            \
    else if (variant == 8)           \
      SGC_D(B_, false, 8);           \
    else if (variant == 9)           \
      SGC_D(B_, false, 12);          \
    else                             \
      SGC_D(B_, false, 0);           \
  } while (0)
      const int nsp = (int)spmm_lane_nsp(op.cols_p, 32 / batch);
      // private accumulator columns: 32 entries per output position per warp
      const size_t per_warp_priv = (size_t)op.ld_out * 32 * sizeof(T);
      int wpb_priv = kBlock / 32;
      while (wpb_priv > 1 && per_warp_priv * wpb_priv > smem_cap) wpb_priv /= 2;
      const size_t smem_priv = per_warp_priv * wpb_priv;
      if (variant == 10 && smem_priv > smem_cap)
        return fail(SGC_ERR_UNSUPPORTED, "SpMM private accumulators do not fit in shared memory");
      switch (batch) {
        case 1: SGC_D2(1); break;
        case 2: SGC_D2(2); break;
        case 4: SGC_D2(4); break;
        case 8: SGC_D2(8); break;
        case 16: SGC_D2(16); break;
        default: SGC_D2(32); break;
      }
#undef SGC_D2
#undef SGC_DP
#undef SGC_D
    } else if (variant >= 3 && batch >= 4) {
      // asynchronous-copy ring of R = 2 (variant 3) or 4 (variant 4) neighbour rows per warp
      const int R = variant == 3 ? 2 : 4;
      const size_t acc_b = ((size_t)batch * op.ld_out * sizeof(T) + 15) & ~(size_t)15;
      const size_t slot_b = (size_t)(batch < 16 ? 16 : batch) + (size_t)op.ld_p * batch * sizeof(T);
      const size_t per_warp_ring = acc_b + R * slot_b;
      int wr = kBlock / 32;
      while (wr > 1 && per_warp_ring * wr > smem_cap) wr /= 2;
      if (per_warp_ring * wr > smem_cap) return fail(SGC_ERR_UNSUPPORTED, "SpMM ring does not fit in shared memory");
      const size_t smem_r = per_warp_ring * wr;
#define SGC_RING(R_)                                                                                         \
  do {                                                                                                       \
    allow_smem(k_spmm_ring<T, R_>, smem_r);                                                                  \
    k_spmm_ring<T, R_><<<grid_for(nitems, wr, 1 << 30), 32 * wr, smem_r, st>>>(                             \
        g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, \
        colors, batch, k, M, (int)op.cols_p, (int)op.ld_p, P, (int)op.ld_out, scratch, tab, si, so);       \
  } while (0)
      if (R == 2) SGC_RING(2);
      else SGC_RING(4);
#undef SGC_RING
    } else
    // a staged table is loaded once per block: a grid of a few blocks per SM, each striding over the rows
    if (pos_bytes == 1)
      launch_spmm_k<T, false, 0, 1>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st,
                                    (int)packed_ld, 16 * num_sms);
    else if (pos_bytes == 2)
      launch_spmm_k<T, false, 0, 2>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st,
                                    (int)packed_ld, 16 * num_sms);
    else if (variant == 1 && per_lane <= 4) SGC_DIRECT_PF(4);
    else if (variant == 1 && per_lane <= 8) SGC_DIRECT_PF(8);
    else if (variant == 1 && per_lane <= 12) SGC_DIRECT_PF(12);
    else launch_spmm_k<T, false, 0>(g, op, batch, k, colors, M, P, scratch, tab, tab_smem, si, so, wpb, smem, st);
#undef SGC_DIRECT_PF
  }
  ++*nk;
  if (g->n_heavy > 0) {
    constexpr int VN = Vec16<T>::n;
    const int64_t width = (int64_t)batch * op.ld_out;
    k_spmm_reduce<T><<<grid_for((int64_t)g->n_heavy * (width / VN), kBlock, 16 * num_sms), kBlock, 0, st>>>(
        g->d_heavy_seg, g->n_heavy, scratch, width, P, width, so);
    ++*nk;
  }
  return SGC_OK;
}

template <typename T, int R, int RPL>
void launch_ema_r(const PlanOp& op, const T* Ma, const T* P, T* out, const uint32_t* tab, int64_t rows, int lb,
                  const ScaleState* sa, const ScaleState* sp, ScaleState* so, cudaStream_t st) {
  const size_t smem = (size_t)(op.cols_a + op.cols_p) * (R + 1) * sizeof(T);
  allow_smem(k_ema<T, R, RPL>, smem);
  const int64_t tiles = (rows + R - 1) / R;
  k_ema<T, R, RPL><<<grid_for(tiles, 1, 1 << 30), kBlock, smem, st>>>(
      Ma, op.ld_a, (int)op.cols_a, P, op.ld_p, (int)op.cols_p, out, op.ld_out, (int)op.cols_out,
      reinterpret_cast<const uint2*>(tab), (int)op.nsplit, op.ema_sym ? 1 : 0, rows, lb, sa, sp, so);
}

// vertex stride (elements) of a staged interleaved row of width ld: a multiple
// of 16 bytes, == batch (mod 32)
inline int ema_vstride(int64_t ld, int batch) {
  const int x = (int)(ld * batch);
  return x + ((batch - x % 32) % 32 + 32) % 32;
}

template <typename T, int B, int RPL>
sgc_status launch_ema_v(const PlanOp& op, const T* Ma, const T* P, T* out, const uint32_t* tab, int64_t nv,
                        const ScaleState* sa, const ScaleState* sp, ScaleState* so, size_t smem_cap,
                        cudaStream_t st) {
  constexpr int V = (32 / B) * RPL;
  const int vsa = ema_vstride(op.ld_a, B), vsp = ema_vstride(op.ld_p, B);
  const size_t buf = ((size_t)V * vsa + (op.ema_sym ? 0 : (size_t)V * vsp)) * sizeof(T);
  const int nbuf = 2 * buf <= smem_cap && 2 * buf <= 100 * 1024 ? 2 : 1;
  if (buf > smem_cap) return fail(SGC_ERR_UNSUPPORTED, "eMA vertex tile does not fit in shared memory");
  const size_t smem = nbuf * buf;
  allow_smem(k_ema_v<T, B, RPL>, smem);
  const int64_t tiles = (nv + V - 1) / V;
  k_ema_v<T, B, RPL><<<grid_for(tiles, 1, 1 << 30), kBlock, smem, st>>>(
      Ma, op.ld_a, (int)op.cols_a, P, op.ld_p, (int)op.cols_p, out, op.ld_out, (int)op.cols_out,
      reinterpret_cast<const uint2*>(tab), (int)op.nsplit, op.ema_sym ? 1 : 0, nv, vsa, vsp, nbuf, sa, sp, so);
  return SGC_OK;
}

sgc_status launch_ema_reg(const PlanOp& op, const float* Ma, const float* P, float* out, int64_t nv, int lb,
                          const ScaleState* sa, const ScaleState* sp, ScaleState* so, cudaStream_t st) {
  const unsigned grid = (unsigned)grid_for(nv << lb, 128, 1 << 30);
#define SGC_ER(K_, AR_, PR_, SYM_)                                                                           \
  if (op.ema_reg_k == K_ && op.a - 1 == AR_ && op.p == PR_ && op.ema_sym == SYM_) {                           \
    k_ema_reg<K_, AR_, PR_, SYM_><<<grid, 128, 0, st>>>(Ma, op.ld_a, P, op.ld_p, out, op.ld_out, nv, lb, sa, sp, \
                                                        so);                                                  \
    return SGC_OK;                                                                                           \
  }
  SGC_EMA_REG_SHAPES(SGC_ER)
#undef SGC_ER
  return fail(SGC_ERR_INTERNAL, "eMA register form not compiled in for this shape");
}

template <typename T, int R>
sgc_status launch_ema_s(const PlanOp& op, const T* Ma, const T* P, T* out, const uint32_t* tab, int64_t nv,
                        const ScaleState* sa, const ScaleState* sp, ScaleState* so, size_t smem_cap, cudaStream_t st) {
  const int elem = (int)sizeof(T);
  const size_t smem = (size_t)ema_sched_smem(R, op.cols_out, op.ld_a, op.ld_p, op.ema_sym, elem, op.ema_upg);
  if (smem > smem_cap) return fail(SGC_ERR_UNSUPPORTED, "scheduled eMA rows do not fit in shared memory");
  allow_smem(k_ema_s<T, R>, smem);
  int dev = 0, nsm = 0, nb = 0;
  SGC_CUDA_TRY(cudaGetDevice(&dev));
  SGC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ema_s<T, R>, 32 * kEmaSchedWarps, smem) != cudaSuccess ||
      nb < 1)
    nb = 1;
  const int64_t tiles = (nv + R - 1) / R;
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)nb * nsm);
  const int G = (int)((op.cols_out + 31) / 32);
  const int rw = (int)ema_sched_rw(op.ld_a, op.ld_p, op.ema_sym);
  k_ema_s<T, R><<<std::max(grid, 1), 32 * kEmaSchedWarps, smem, st>>>(Ma, op.ld_a, P, op.ld_p, out, op.ld_out, tab, G, op.ema_upg,
                                                         op.ema_sym ? 1 : 0, op.ema_sym ? 0 : (int)op.ld_a, rw, nv,
                                                         (int)op.nsplit, sa, sp, so);
  return SGC_OK;
}

template <typename T>
sgc_status launch_ema(const PlanOp& op, const T* Ma, const T* P, T* out, const uint32_t* tab, int64_t rows, int lb,
                      const ScaleState* sa, const ScaleState* sp, ScaleState* so, size_t smem_cap, cudaStream_t st) {
  if (op.ema_sched > 0) {
    if (lb != 0) return fail(SGC_ERR_INTERNAL, "the scheduled eMA takes one coloring per pass");
    switch (op.ema_sched) {
      case 12: return launch_ema_s<T, 12>(op, Ma, P, out, tab, rows, sa, sp, so, smem_cap, st);
      case 8: return launch_ema_s<T, 8>(op, Ma, P, out, tab, rows, sa, sp, so, smem_cap, st);
      case 6: return launch_ema_s<T, 6>(op, Ma, P, out, tab, rows, sa, sp, so, smem_cap, st);
      case 4: return launch_ema_s<T, 4>(op, Ma, P, out, tab, rows, sa, sp, so, smem_cap, st);
      default: return launch_ema_s<T, 2>(op, Ma, P, out, tab, rows, sa, sp, so, smem_cap, st);
    }
  }
  if (op.ema_reg_k > 0) {
    if constexpr (std::is_same<T, float>::value)
      return launch_ema_reg(op, Ma, P, out, rows >> lb, lb, sa, sp, so, st);
    else
      return fail(SGC_ERR_INTERNAL, "the register-form eMA is FP32 only");
  }
  if (op.ema_vrpl > 0) {
    const int64_t nv = rows >> lb;
    const int B = 1 << lb;
#define SGC_EV(B_)                                                                                \
  return op.ema_vrpl == 2 ? launch_ema_v<T, B_, 2>(op, Ma, P, out, tab, nv, sa, sp, so, smem_cap, st) \
                          : launch_ema_v<T, B_, 1>(op, Ma, P, out, tab, nv, sa, sp, so, smem_cap, st)
    switch (B) {
      case 4: SGC_EV(4);
      case 8: SGC_EV(8);
      case 16: SGC_EV(16);
      case 32: SGC_EV(32);
      default: return fail(SGC_ERR_INTERNAL, "eMA vertex tiles need 4..32 colorings per pass");
    }
#undef SGC_EV
  }
  switch (op.ema_rows) {
    case 64: launch_ema_r<T, 64, 2>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    case 32: launch_ema_r<T, 32, 1>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    case 16: launch_ema_r<T, 16, 1>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    case 8: launch_ema_r<T, 8, 1>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    case 4: launch_ema_r<T, 4, 1>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    case 2: launch_ema_r<T, 2, 1>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    case 1: launch_ema_r<T, 1, 1>(op, Ma, P, out, tab, rows, lb, sa, sp, so, st); break;
    default:  // rows too wide to stage: operands through L1 (the table holds raw indices)
      k_ema_gl<T><<<grid_for(rows, kBlock / 32, 1 << 30), kBlock, 0, st>>>(
          Ma, op.ld_a, P, op.ld_p, out, op.ld_out, (int)op.cols_out, reinterpret_cast<const uint2*>(tab),
          (int)op.nsplit, op.ema_sym ? 1 : 0, rows, lb, sa, sp, so);
      break;
  }
  return SGC_OK;
}

int profile_slot(Profiler* prof, const PlanOp& op, int batch, int k) {
  for (size_t i = 0; i < prof->agg.size(); ++i) {
    const OpProfile& a = prof->agg[i];
    if (a.kind == op.kind && a.t == op.t && a.a == op.a && a.p == op.p && a.batch == batch && a.k == k)
      return (int)i;
  }
  OpProfile a;
  a.k = k;
  a.kind = op.kind;
  a.t = op.t;
  a.a = op.a;
  a.p = op.p;
  a.batch = batch;
  a.bytes = op.alg_bytes;
  a.flops = op.alg_flops;
  a.gather = op.gather_bytes;
  prof->agg.push_back(a);
  return (int)prof->agg.size() - 1;
}

// The grouped SpMM: the color-grouped neighbour lists of the pass (built by the
// first grouped op), then a warp per (item, coloring) with the chunk width
// 32 * NR closest above the row width (at most 512 columns per chunk, or 256 for
// op.spmm_variant == 15: fewer registers, more warps), then
// the heavy rows' segment partials summed.  Chunks of at most 512 columns keep two neighbours'
// rows and the sums in registers at 4 warps of 8 per SM's register file.
template <typename T>
sgc_status launch_spmm_grouped(const sgc_graph* g, const Plan& plan, const PlanOp& op, int batch,
                               const uint8_t* colors, const T* M, T* P, T* scratch, const uint32_t* tab,
                               int32_t* gids, uint8_t* gcols, int32_t* gkept, bool* ready, const ScaleState* si,
                               ScaleState* so, int num_sms, size_t smem_cap, cudaStream_t st, int64_t* nk) {
  if (batch != 1 && batch != 2 && batch != 4) return fail(SGC_ERR_INTERNAL, "grouped SpMM: 1, 2 or 4 colorings per pass");
  if (plan.k > 32 || op.ld_out >= 65535) return fail(SGC_ERR_INTERNAL, "grouped SpMM: shape out of range");
  if (plan.buf_gids < 0 || plan.buf_gcols < 0 || plan.buf_gkept < 0)
    return fail(SGC_ERR_INTERNAL, "grouped SpMM: the plan has no neighbour-group buffers");
  const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
  const int wpb = kBlock / 32;
  if (!*ready) {
    const unsigned grid = (unsigned)grid_for(nitems * batch, wpb, 1 << 30);
#define SGC_GN(B_)                                                                                             \
  k_group_nbrs<B_><<<grid, kBlock, 0, st>>>(g->d_row_ptr, g->d_col_idx, g->n_seg, g->d_seg_row, g->d_seg_lo, \
                                             g->d_seg_hi, g->n_heavy, g->n_act, colors, g->nnz, gids, gcols,   \
                                             gkept)
    if (batch == 1) SGC_GN(1);
    else if (batch == 2) SGC_GN(2);
    else SGC_GN(4);
#undef SGC_GN
    ++*nk;
    *ready = true;
  }
  if (op.spmm_variant == 16 || op.spmm_variant == 17) {
    // the staged form: one block per SM of as many warps (at most 16) as shared memory holds
    if constexpr (std::is_same<T, float>::value) {
      if (batch != 1) return fail(SGC_ERR_INTERNAL, "staged SpMM: one coloring per pass");
      const int nr4 = spmm_staged_nr4(op.cols_p, op.spmm_variant), rs = spmm_staged_rs(op.spmm_variant);
      const size_t pw = (size_t)spmm_staged_warp_bytes(op.cols_p, op.ld_out, op.spmm_variant);
      const int wn = (int)std::min<size_t>(16, smem_cap / pw);
      if (wn < 2) return fail(SGC_ERR_UNSUPPORTED, "staged SpMM: two warps' rings do not fit in shared memory");
      if (reinterpret_cast<uintptr_t>(M) % 16 || reinterpret_cast<uintptr_t>(tab) % 16 ||
          reinterpret_cast<uintptr_t>(P) % 16 || reinterpret_cast<uintptr_t>(scratch) % 16 || op.ld_p % 4 ||
          op.ld_out % 4)
        return fail(SGC_ERR_INTERNAL, "staged SpMM: rows and tables must start on 16-byte boundaries");
      const size_t smem = pw * wn;
      const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms, (nitems + wn - 1) / wn));
      const uint16_t* tab16 = reinterpret_cast<const uint16_t*>(tab);
      const int wpitch = (int)spmm_staged_pitch(op.cols_p);
#define SGC_GS(NR4_, RS_)                                                                                    \
  do {                                                                                                       \
    allow_smem(k_spmm_gs<NR4_, RS_>, smem);                                                                  \
    k_spmm_gs<NR4_, RS_><<<grid, 32 * wn, smem, st>>>(g->d_row_ptr, g->n_seg, g->d_seg_row, g->d_seg_lo,    \
                                                      g->d_seg_hi, g->n_heavy, g->n_act, colors, plan.k, gids, \
                                                      gcols, gkept, M, (int)op.cols_p, (int)op.ld_p, P,      \
                                                      (int)op.ld_out, scratch, tab16, wpitch, si, so);       \
  } while (0)
      if (rs == 2) {
        if (nr4 == 2) SGC_GS(2, 2);
        else if (nr4 == 4) SGC_GS(4, 2);
        else SGC_GS(8, 2);
      } else {
        if (nr4 == 2) SGC_GS(2, 3);
        else if (nr4 == 4) SGC_GS(4, 3);
        else SGC_GS(8, 3);
      }
#undef SGC_GS
      ++*nk;
    } else {
      return fail(SGC_ERR_INTERNAL, "staged SpMM: FP32 tables only");
    }
  } else {
  const size_t per_warp = (size_t)op.ld_out * sizeof(T);
  int w = wpb;
  while (w > 2 && per_warp * w > smem_cap) w /= 2;
  if (per_warp * w > smem_cap) return fail(SGC_ERR_UNSUPPORTED, "grouped SpMM: output row does not fit in shared memory");
  const size_t smem = per_warp * w;
  const int w_in = (int)op.cols_p;
  const int need = (w_in + 31) / 32;
  const int nr_cap = op.spmm_variant == 15 ? 8 : 16;  // wider rows: chunks of 32 * nr_cap columns
  const int nr = std::min(nr_cap, need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 16);
  const uint16_t* tab16 = reinterpret_cast<const uint16_t*>(tab);
  const unsigned grid = (unsigned)grid_for(nitems * batch, w, 1 << 30);
#define SGC_G(B_, NR_)                                                                                          \
  do {                                                                                                          \
    allow_smem(k_spmm_g<T, B_, NR_>, smem);                                                                     \
    k_spmm_g<T, B_, NR_><<<grid, 32 * w, smem, st>>>(g->d_row_ptr, g->n_seg, g->d_seg_row, g->d_seg_lo,        \
                                                     g->d_seg_hi, g->n_heavy, g->n_act, colors, plan.k, g->nnz, \
                                                     gids, gcols, gkept, M, w_in, (int)op.ld_p, P,             \
                                                     (int)op.ld_out, scratch, tab16, si, so);                   \
  } while (0)
#define SGC_G2(B_)                      \
  do {                                  \
    switch (nr) {                       \
      case 2: SGC_G(B_, 2); break;      \
      case 4: SGC_G(B_, 4); break;      \
      case 8: SGC_G(B_, 8); break;      \
      default: SGC_G(B_, 16); break;    \
    }                                   \
  } while (0)
  if (batch == 1) SGC_G2(1);
  else if (batch == 2) SGC_G2(2);
  else SGC_G2(4);
#undef SGC_G2
#undef SGC_G
  ++*nk;
  }
  if (g->n_heavy > 0) {
    constexpr int VN = Vec16<T>::n;
    const int64_t width = (int64_t)batch * op.ld_out;
    k_spmm_reduce<T><<<grid_for((int64_t)g->n_heavy * (width / VN), kBlock, 16 * num_sms), kBlock, 0, st>>>(
        g->d_heavy_seg, g->n_heavy, scratch, width, P, width, so);
    ++*nk;
  }
  return SGC_OK;
}

template <typename T>
sgc_status run_pass_t(const sgc_graph* g, const Plan& plan, const uint32_t* d_tabs, char* ws, cudaStream_t st,
                      Profiler* prof, int64_t* kernels) {
  int dev = 0, num_sms = 0, smem_optin = 0;
  SGC_CUDA_TRY(cudaGetDevice(&dev));
  SGC_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  SGC_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t smem_cap = (size_t)smem_optin;
  auto buf = [&](int b) -> char* { return ws + plan.bufs[b].offset; };
  const int B = plan.batch;
  const int64_t rows = plan.rows;
  ScaleState* states = reinterpret_cast<ScaleState*>(buf(plan.buf_states));
  auto S = [&](int i) -> ScaleState* { return i < 0 ? nullptr : states + i; };
  const uint8_t* colors = reinterpret_cast<const uint8_t*>(buf(plan.buf_colors));
  T* scratch = reinterpret_cast<T*>(buf(plan.buf_scratch));
  double* partials = reinterpret_cast<double*>(buf(plan.buf_partials));
  double* outv = reinterpret_cast<double*>(buf(plan.buf_out));
  const bool fp32 = std::is_same<T, float>::value;
  int lb = 0;
  while ((1 << lb) < B) ++lb;
  if ((1 << lb) != B || B > 32) return fail(SGC_ERR_INTERNAL, "batch must be a power of two <= 32");

  if (fp32) SGC_CUDA_TRY(cudaMemsetAsync(states, 0, sizeof(ScaleState) * (size_t)std::max(1, plan.n_states), st));
  int64_t nk = 0;
  bool grouped_ready = false;  // neighbour lists grouped by color (once per pass, before the first grouped SpMM)
  for (size_t oi = 0; oi < plan.ops.size(); ++oi) {
    const PlanOp& op = plan.ops[oi];
    int slot = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int64_t nk0 = nk;
    if (prof) {
      if (prof->by_index) {
        if (prof->agg.size() < plan.ops.size()) prof->agg.resize(plan.ops.size());
        slot = (int)oi;
      } else {
        slot = profile_slot(prof, op, B, plan.k);
      }
      SGC_CUDA_TRY(cudaEventCreate(&e0));
      SGC_CUDA_TRY(cudaEventCreate(&e1));
      SGC_CUDA_TRY(cudaEventRecord(e0, st));
    }
    switch (op.kind) {
      case OP_COLOR:
        k_color<<<grid_for(rows, kBlock, 8 * num_sms), kBlock, 0, st>>>(
            g->d_orig, g->n_act, B, reinterpret_cast<const uint64_t*>(buf(plan.buf_seeds)), plan.k,
            reinterpret_cast<uint8_t*>(buf(plan.buf_colors)));
        ++nk;
        break;
      case OP_HIST: {
        T* H = reinterpret_cast<T*>(buf(op.out));
        int32_t* hh = reinterpret_cast<int32_t*>(buf(plan.buf_hist_heavy));
        if (g->n_heavy > 0)
          SGC_CUDA_TRY(cudaMemsetAsync(hh, 0, sizeof(int32_t) * (size_t)g->n_heavy * B * plan.k, st));
        const int64_t nitems = (int64_t)g->n_seg + (g->n_act - g->n_heavy);
        const size_t smem = (size_t)(kBlock / 32) * B * plan.k * sizeof(int32_t);
        const unsigned hgrid = (unsigned)grid_for(nitems, kBlock / 32, 1 << 30);
#define SGC_HIST(B_)                                                                                          \
  do {                                                                                                        \
    allow_smem(k_hist<T, B_>, smem);                                                                          \
    k_hist<T, B_><<<hgrid, kBlock, smem, st>>>(g->d_row_ptr, g->d_col_idx, colors, plan.k, g->n_seg,          \
                                               g->d_seg_row, g->d_seg_lo, g->d_seg_hi, g->n_heavy, g->n_act, H, \
                                               op.ld_out, hh, S(op.state_out));                               \
  } while (0)
        switch (B) {
          case 1: SGC_HIST(1); break;
          case 2: SGC_HIST(2); break;
          case 4: SGC_HIST(4); break;
          case 8: SGC_HIST(8); break;
          case 16: SGC_HIST(16); break;
          case 32: SGC_HIST(32); break;
          default: return fail(SGC_ERR_INTERNAL, "colorings per pass must be a power of two up to 32");
        }
#undef SGC_HIST
        ++nk;
        if (g->n_heavy > 0) {
          k_hist_heavy_out<T><<<grid_for((int64_t)g->n_heavy * B * op.ld_out, kBlock, 8 * num_sms), kBlock, 0, st>>>(
              hh, colors, g->n_heavy, B, plan.k, H, op.ld_out, S(op.state_out));
          ++nk;
        }
        break;
      }
      case OP_SPMM: {
        if (op.spmm_variant == 14) {
          const int64_t items = rows * op.ld_out;
          k_spmm_col<T><<<grid_for(items, kBlock, 64 * num_sms), kBlock, 0, st>>>(
              g->d_row_ptr, g->d_col_idx, g->n_act, colors, lb, plan.k, reinterpret_cast<const T*>(buf(op.in_p)),
              op.ld_p, reinterpret_cast<T*>(buf(op.out)), op.ld_out, (int)op.cols_out, d_tabs + op.tab_off,
              S(op.state_p), S(op.state_out));
          ++nk;
          break;
        }
        if (spmm_variant_grouped(op.spmm_variant)) {
          sgc_status rc = launch_spmm_grouped<T>(g, plan, op, B, colors, reinterpret_cast<const T*>(buf(op.in_p)),
                                                 reinterpret_cast<T*>(buf(op.out)), scratch, d_tabs + op.tab_off,
                                                 reinterpret_cast<int32_t*>(buf(plan.buf_gids)),
                                                 reinterpret_cast<uint8_t*>(buf(plan.buf_gcols)),
                                                 reinterpret_cast<int32_t*>(buf(plan.buf_gkept)), &grouped_ready,
                                                 S(op.state_p), S(op.state_out), num_sms, smem_cap, st, &nk);
          if (rc != SGC_OK) return rc;
          break;
        }
        sgc_status rc = launch_spmm<T>(g, op, B, plan.k, colors, reinterpret_cast<const T*>(buf(op.in_p)),
                                       reinterpret_cast<T*>(buf(op.out)), scratch, d_tabs + op.tab_off,
                                       S(op.state_p), S(op.state_out), num_sms, smem_cap, st, &nk);
        if (rc != SGC_OK) return rc;
        break;
      }
      case OP_EMA: {
        if (op.ema_final) {
          if constexpr (std::is_same<T, float>::value) {
            bool done = false;
#define SGC_EF(K_, PR_)                                                                                          \
  if (!done && op.ema_reg_k == K_ && op.p == PR_) {                                                              \
    int nb = 0;                                                                                                  \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ema_final_reg<K_, PR_>, 128, 0) != cudaSuccess ||   \
        nb < 1)                                                                                                  \
      nb = 1;                                                                                                    \
    const int grid = std::min(plan.final_blocks, nb * num_sms);                                                  \
    SGC_CUDA_TRY(cudaMemsetAsync(partials, 0, sizeof(double) * (size_t)plan.final_blocks * B, st));              \
    k_ema_final_reg<K_, PR_><<<grid, 128, 0, st>>>(reinterpret_cast<const float*>(buf(op.in_p)), op.ld_p, rows,  \
                                                   lb, S(op.state_p), S(op.state_out), partials);               \
    done = true;                                                                                                 \
  }
            SGC_EMA_FINAL_SHAPES(SGC_EF)
#undef SGC_EF
            if (!done) return fail(SGC_ERR_INTERNAL, "fused eMA + last step not compiled in for this shape");
            ++nk;
            break;
          } else {
            return fail(SGC_ERR_INTERNAL, "the fused eMA + last step is FP32 only");
          }
        }
        sgc_status rc = launch_ema<T>(op, reinterpret_cast<const T*>(buf(op.in_a)),
                                      reinterpret_cast<const T*>(buf(op.in_p)), reinterpret_cast<T*>(buf(op.out)),
                                      d_tabs + op.tab_off, rows, lb, S(op.state_a), S(op.state_p), S(op.state_out),
                                      smem_cap, st);
        if (rc != SGC_OK) return rc;
        ++nk;
        break;
      }
      case OP_FINAL_LEAF:
        k_final_leaf<T><<<plan.final_blocks, kBlock, 0, st>>>(reinterpret_cast<const T*>(buf(op.in_p)), op.ld_p, rows,
                                                              lb, partials);
        k_final_sum<<<1, 32, 0, st>>>(partials, plan.final_blocks, B, nullptr, S(op.state_p), fp32 ? 1 : 0, outv);
        nk += 2;
        break;
      case OP_UNPRUNED: {
        const int64_t items = rows * op.ld_out;
        k_unpruned<T><<<grid_for(items, kBlock, 64 * num_sms), kBlock, 0, st>>>(
            g->d_row_ptr, g->d_col_idx, g->n_act, colors, lb, plan.k,
            op.in_a >= 0 ? reinterpret_cast<const T*>(buf(op.in_a)) : nullptr, op.ld_a,
            op.in_p >= 0 ? reinterpret_cast<const T*>(buf(op.in_p)) : nullptr, op.ld_p, (int)op.cols_p,
            reinterpret_cast<T*>(buf(op.out)), op.ld_out, (int)op.cols_out,
            reinterpret_cast<const uint2*>(d_tabs + op.tab_off), (int)op.nsplit, d_tabs + op.tab2_off, g->max_deg,
            S(op.state_a), S(op.state_p), S(op.state_out));
        ++nk;
        break;
      }
      case OP_FINAL_SUM:
        k_final_rows<T><<<plan.final_blocks, kBlock, 0, st>>>(reinterpret_cast<const T*>(buf(op.in_p)), op.ld_p,
                                                              (int)op.cols_p, rows, lb, partials);
        k_final_sum<<<1, 32, 0, st>>>(partials, plan.final_blocks, B, nullptr, S(op.state_p), fp32 ? 1 : 0, outv);
        nk += 2;
        break;
      case OP_FINAL: {
        bool done = op.final_fused;  // the fused eMA wrote the partials
#define SGC_FR(K_, PR_)                                                                                      \
  if (!done && op.final_reg && plan.k - 1 == K_ && op.p == PR_) {                                            \
    k_final_reg<T, K_, PR_><<<plan.final_blocks, kBlock, 0, st>>>(reinterpret_cast<const T*>(buf(op.in_a)),  \
                                                                  op.ld_a, reinterpret_cast<const T*>(buf(op.in_p)), \
                                                                  op.ld_p, rows, lb, partials);                \
    done = true;                                                                                             \
  }
        SGC_FINAL_REG_SHAPES(SGC_FR)
#undef SGC_FR
        if (!done)
          k_final<T><<<plan.final_blocks, kBlock, 0, st>>>(reinterpret_cast<const T*>(buf(op.in_a)), op.ld_a,
                                                           reinterpret_cast<const T*>(buf(op.in_p)), op.ld_p,
                                                           (int)op.cols_p, d_tabs + op.tab_off, rows, lb, partials);
      }
        k_final_sum<<<1, 32, 0, st>>>(partials, plan.final_blocks, B, S(op.state_a), S(op.state_p), fp32 ? 1 : 0,
                                      outv);
        nk += op.final_fused ? 1 : 2;  // fused: the partials came from the eMA's kernel
        break;
    }
    if (prof) {
      SGC_CUDA_TRY(cudaEventRecord(e1, st));
      prof->pending.push_back({slot, e0, e1});
      prof->agg[slot].launches += 1;
      prof->agg[slot].kernels += nk - nk0;
    }
  }
  SGC_CUDA_TRY(cudaGetLastError());
  if (kernels) *kernels += nk;
  return SGC_OK;
}

}  // namespace

bool ema_final_compiled(int K, int p) {
#define SGC_EF(K_, PR_) \
  if (K == K_ && p == PR_) return true;
  SGC_EMA_FINAL_SHAPES(SGC_EF)
#undef SGC_EF
  return false;
}

bool final_reg_compiled(int K, int p) {
#define SGC_FR(K_, PR_) \
  if (K == K_ && p == PR_) return true;
  SGC_FINAL_REG_SHAPES(SGC_FR)
#undef SGC_FR
  return false;
}

bool ema_reg_compiled(int K, int a_minus_1, int p, bool sym) {
#define SGC_ER(K_, AR_, PR_, SYM_) \
  if (K == K_ && a_minus_1 == AR_ && p == PR_ && sym == SYM_) return true;
  SGC_EMA_REG_SHAPES(SGC_ER)
#undef SGC_ER
  return false;
}

sgc_status run_pass(const sgc_graph* g, const Plan& plan, const uint32_t* d_tabs, char* ws, cudaStream_t stream,
                    Profiler* prof, int64_t* kernels) {
  if (plan.precision == SGC_FP64) return run_pass_t<double>(g, plan, d_tabs, ws, stream, prof, kernels);
  return run_pass_t<float>(g, plan, d_tabs, ws, stream, prof, kernels);
}

}  // namespace sgc
