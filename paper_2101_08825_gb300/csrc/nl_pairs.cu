// nl_pairs.cu -- element-pair search (Sec. 5, eq. k_l with Sec. 5.1 eq. mindist) and the
// CSR sparsity pattern of the stiffness matrix, plus the scan used by both.
//
// Pairs: elements are binned by the centres of their bounding boxes into a uniform grid
// whose cell side s is at least delta + eps + the largest box side, so that a pair with
// aprx-min-dist < delta + eps has centres less than s apart on every axis and lies in
// neighbouring cells.  A count pass (one warp per inner element m) is followed by a scan
// and a fill pass (one CTA per m) that collects, sorts (bitonic, in shared memory) and
// writes the l of every pair of m.  The box test is screened in FP32 on boxes rounded
// outwards and decided by the exact FP64 expression of eq. (mindist) wherever the screened
// distance lies within a margin of the threshold, so the list is bit-identical to a plain
// FP64 evaluation.
//
// Pattern: row i holds the nodes of every l with (m, l) in J and i a node of m.  One CTA
// per row gathers the union of the l over the elements m around i in a shared-memory hash
// set, then the nodes of those l in a second set, and (fill pass) sorts them.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "nl_internal.h"

namespace nlx {

// ---- scan ---------------------------------------------------------------------------------
namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__global__ void k_tile_sums(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t ws[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += (int64_t)in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of one tile with a per-tile offset; out[n] = total by the last tile.
template <typename T>
__global__ void k_tile_scan(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                            int64_t* __restrict__ out) {
  __shared__ int64_t ws[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t i = base + k;
    v[k] = (i < n) ? (int64_t)in[i] : 0;
    s += v[k];
  }
  // inclusive scan of the per-thread sums across the block
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int64_t wpre = 0;
  for (int k = 0; k < w; k++) wpre += ws[k];
  int64_t run = (offs ? offs[blockIdx.x] : 0) + wpre + inc - s;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
    if (i == n - 1) out[n] = run;
  }
}

template <typename T>
nl_status scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    NL_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return NL_OK;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    k_tile_scan<T><<<NL_CNT(1), SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
    NL_CUDA(cudaGetLastError());
    return NL_OK;
  }
  DevBuf<int64_t> sums, offs;
  NL_TRY(sums.alloc(tiles, s));
  NL_TRY(offs.alloc(tiles + 1, s));
  k_tile_sums<T><<<NL_CNT((unsigned)tiles), SCAN_THREADS, 0, s>>>(in, n, sums.p);
  NL_CUDA(cudaGetLastError());
  NL_TRY(scan_impl<int64_t>(sums.p, offs.p, tiles, s));
  k_tile_scan<T><<<NL_CNT((unsigned)tiles), SCAN_THREADS, 0, s>>>(in, n, offs.p, out);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}
}  // namespace

nl_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, s);
}
nl_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, s);
}

// ---- pair search ----------------------------------------------------------------------------
namespace {

constexpr int ERR_PAIR_COUNT = 1;    // fill pass found a different number of pairs
constexpr int ERR_HASH_FULL = 2;     // a shared-memory hash set overflowed
constexpr int ERR_ROW_COUNT = 4;     // row fill pass found a different number of columns

struct Grid {
  double lo[3];
  double inv_s;
  int n[3];
};

template <int D>
__device__ __forceinline__ void cell_of(const Grid& g, const double* lo, const double* hi, int* c) {
  for (int k = 0; k < D; k++) {
    double ctr = 0.5 * (lo[k] + hi[k]);
    int v = (int)floor((ctr - g.lo[k]) * g.inv_s);
    c[k] = min(max(v, 0), g.n[k] - 1);
  }
}

template <int D>
__device__ __forceinline__ int cell_id(const Grid& g, const int* c) {
  int id = c[D - 1];
  for (int k = D - 2; k >= 0; k--) id = id * g.n[k] + c[k];
  return id;
}

// eq. (mindist) for boxes (lo1, hi1) of E_l and (lo2, hi2) of E_m, compared with delta + eps.
template <int D>
__device__ __forceinline__ bool in_reach(const double* lo1, const double* hi1, const double* lo2,
                                         const double* hi2, double reach) {
  double m = 0.0;
#pragma unroll
  for (int k = 0; k < D; k++) {
    double d1 = __dsub_rn(lo1[k], hi2[k]);
    double d2 = __dsub_rn(lo2[k], hi1[k]);
    double t = d1 > d2 ? d1 : d2;
    m = t > m ? t : m;
  }
  return m < reach;
}

// The same test screened in FP32 on boxes rounded outwards (fbox: lo rounded down, hi rounded
// up, so the FP32 box contains the FP64 one): a screened distance below reach - margin or
// above reach + margin decides; in between the FP64 test of eq. (mindist) decides.  margin
// bounds the rounding of the FP32 boxes and of the FP32 subtraction, so the result is that of
// the FP64 test for every pair.
struct Screen {
  const float* flo;  // [n_elem][D] lower box corners rounded down
  const float* fhi;  // [n_elem][D] upper box corners rounded up
  float lo_t, hi_t;  // reach - margin, reach + margin
};

template <int D>
__device__ __forceinline__ bool in_reach_screened(const Screen& S, int64_t l, const float* flo_m,
                                                  const float* fhi_m, const double* __restrict__ blo,
                                                  const double* __restrict__ bhi, const double* lo_m,
                                                  const double* hi_m, double reach) {
  float mf = 0.f;
#pragma unroll
  for (int k = 0; k < D; k++) {
    const float d1 = S.flo[l * D + k] - fhi_m[k];
    const float d2 = flo_m[k] - S.fhi[l * D + k];
    mf = fmaxf(mf, fmaxf(d1, d2));
  }
  if (mf < S.lo_t) return true;
  if (mf > S.hi_t) return false;
  double lo_l[D], hi_l[D];
#pragma unroll
  for (int k = 0; k < D; k++) {
    lo_l[k] = blo[l * D + k];
    hi_l[k] = bhi[l * D + k];
  }
  return in_reach<D>(lo_l, hi_l, lo_m, hi_m, reach);
}

__global__ void k_round_boxes(int64_t n, const double* __restrict__ blo, const double* __restrict__ bhi,
                              float* __restrict__ flo, float* __restrict__ fhi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  flo[i] = __double2float_rd(blo[i]);
  fhi[i] = __double2float_ru(bhi[i]);
}

template <int D>
__global__ void k_bin_count(int64_t n_elem, Grid g, const double* __restrict__ blo,
                            const double* __restrict__ bhi, int32_t* __restrict__ cell_cnt) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  int c[3];
  cell_of<D>(g, blo + e * D, bhi + e * D, c);
  atomicAdd(&cell_cnt[cell_id<D>(g, c)], 1);
}

template <int D>
__global__ void k_bin_fill(int64_t n_elem, Grid g, const double* __restrict__ blo,
                           const double* __restrict__ bhi, const int64_t* __restrict__ cell_off,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ items) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  int c[3];
  cell_of<D>(g, blo + e * D, bhi + e * D, c);
  int id = cell_id<D>(g, c);
  int pos = atomicAdd(&cursor[id], 1);
  items[cell_off[id] + pos] = (int32_t)e;
}

template <int D>
__global__ void k_pairs_count(int64_t n_elem, Grid g, double reach, const double* __restrict__ blo,
                              const double* __restrict__ bhi, const int64_t* __restrict__ cell_off,
                              const int32_t* __restrict__ items, int64_t* __restrict__ cnt,
                              int32_t* __restrict__ max_cnt, Screen S) {
  int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (m >= n_elem) return;
  double lo_m[D], hi_m[D];
  for (int k = 0; k < D; k++) {
    lo_m[k] = blo[m * D + k];
    hi_m[k] = bhi[m * D + k];
  }
  float flo_m[D], fhi_m[D];
  for (int k = 0; k < D; k++) {
    flo_m[k] = S.flo[m * D + k];
    fhi_m[k] = S.fhi[m * D + k];
  }
  int c[3];
  cell_of<D>(g, lo_m, hi_m, c);
  int64_t count = 0;
  const int nb = (D == 2) ? 9 : 27;
  for (int b = 0; b < nb; b++) {
    int cc[3] = {c[0] + b % 3 - 1, c[1] + (b / 3) % 3 - 1, (D == 3) ? c[2] + b / 9 - 1 : 0};
    bool ok = true;
    for (int k = 0; k < D; k++) ok &= cc[k] >= 0 && cc[k] < g.n[k];
    if (!ok) continue;
    int id = cell_id<D>(g, cc);
    for (int64_t t = cell_off[id] + lane; t < cell_off[id + 1]; t += 32) {
      const int32_t l = items[t];
      count += in_reach_screened<D>(S, l, flo_m, fhi_m, blo, bhi, lo_m, hi_m, reach) ? 1 : 0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
  if (lane == 0) {
    cnt[m] = count;
    atomicMax(max_cnt, (int32_t)count);
  }
}

// Bitonic sort of n (a power of two) ints in shared memory by the whole block.
__device__ void block_bitonic_sort(int32_t* a, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          int32_t x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

template <int D>
__global__ void k_pairs_fill(int64_t n_elem, Grid g, double reach, const double* __restrict__ blo,
                             const double* __restrict__ bhi, const int64_t* __restrict__ cell_off,
                             const int32_t* __restrict__ items, const int64_t* __restrict__ pair_off,
                             int32_t* __restrict__ pair_l, int cap, int* __restrict__ err, Screen S) {
  extern __shared__ int32_t buf[];
  __shared__ int nfound;
  int64_t m = blockIdx.x;
  if (threadIdx.x == 0) nfound = 0;
  __syncthreads();
  double lo_m[D], hi_m[D];
  for (int k = 0; k < D; k++) {
    lo_m[k] = blo[m * D + k];
    hi_m[k] = bhi[m * D + k];
  }
  float flo_m[D], fhi_m[D];
  for (int k = 0; k < D; k++) {
    flo_m[k] = S.flo[m * D + k];
    fhi_m[k] = S.fhi[m * D + k];
  }
  int c[3];
  cell_of<D>(g, lo_m, hi_m, c);
  const int nb = (D == 2) ? 9 : 27;
  for (int b = 0; b < nb; b++) {
    int cc[3] = {c[0] + b % 3 - 1, c[1] + (b / 3) % 3 - 1, (D == 3) ? c[2] + b / 9 - 1 : 0};
    bool ok = true;
    for (int k = 0; k < D; k++) ok &= cc[k] >= 0 && cc[k] < g.n[k];
    if (!ok) continue;
    int id = cell_id<D>(g, cc);
    for (int64_t t = cell_off[id] + threadIdx.x; t < cell_off[id + 1]; t += blockDim.x) {
      const int32_t l = items[t];
      if (in_reach_screened<D>(S, l, flo_m, fhi_m, blo, bhi, lo_m, hi_m, reach)) {
        int pos = atomicAdd(&nfound, 1);
        if (pos < cap) buf[pos] = l;
      }
    }
  }
  __syncthreads();
  int n = nfound;
  int64_t expect = pair_off[m + 1] - pair_off[m];
  if (n != expect || n > cap) {
    if (threadIdx.x == 0) atomicOr(err, ERR_PAIR_COUNT);
    return;
  }
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int i = n + threadIdx.x; i < np2; i += blockDim.x) buf[i] = INT_MAX;
  __syncthreads();
  block_bitonic_sort(buf, np2);
  for (int i = threadIdx.x; i < n; i += blockDim.x) pair_l[pair_off[m] + i] = buf[i];
}

// ---- pattern ----------------------------------------------------------------------------------
__device__ __forceinline__ int hash_insert(int32_t* tab, int mask, int32_t key, int* overflow) {
  uint32_t h = ((uint32_t)key * 2654435761u) & (uint32_t)mask;
  for (int probe = 0; probe <= mask; probe++) {
    int32_t old = atomicCAS(&tab[h], -1, key);
    if (old == -1) return 1;
    if (old == key) return 0;
    h = (h + 1) & (uint32_t)mask;
  }
  *overflow = 1;
  return 0;
}

__global__ void k_row_bound(int64_t n_vert, const int64_t* __restrict__ n2e_off,
                            const int32_t* __restrict__ n2e, const int64_t* __restrict__ pair_off,
                            int64_t* __restrict__ max_sum) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_vert) return;
  int64_t s = 0;
  for (int64_t t = n2e_off[i]; t < n2e_off[i + 1]; t++) {
    int32_t m = n2e[t];
    s += pair_off[m + 1] - pair_off[m];
  }
  atomicMax((unsigned long long*)max_sum, (unsigned long long)s);
}

// MODE 0: count the columns of row i; MODE 1: write them sorted into col at row_ptr[i];
// MODE 2: count them and write them sorted into the staging rows tmp[i * rowcap ...] (one pass
// instead of two; k_copy_rows then packs the staged rows once row_ptr is known).
// conn holds nb nodes per element (the vertices, then a P2 element's edge nodes).
template <int D, int MODE>
__global__ void k_rows(int64_t n_vert, const int32_t* __restrict__ conn, int nb,
                       const int64_t* __restrict__ n2e_off, const int32_t* __restrict__ n2e,
                       const int64_t* __restrict__ pair_off, const int32_t* __restrict__ pair_l,
                       int eh, int nh, int32_t* __restrict__ row_cnt,
                       const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                       int* __restrict__ err, int* __restrict__ max_row, int32_t* __restrict__ tmp,
                       int rowcap) {
  constexpr bool FILL = MODE == 1;
  extern __shared__ int32_t smem[];
  int32_t* etab = smem;
  int32_t* ntab = smem + eh;
  __shared__ int ncount, overflow;
  int64_t i = blockIdx.x;
  for (int t = threadIdx.x; t < eh + nh; t += blockDim.x) smem[t] = -1;
  if (threadIdx.x == 0) {
    ncount = 0;
    overflow = 0;
  }
  __syncthreads();
  for (int64_t t = n2e_off[i]; t < n2e_off[i + 1]; t++) {
    int32_t m = n2e[t];
    for (int64_t p = pair_off[m] + threadIdx.x; p < pair_off[m + 1]; p += blockDim.x)
      hash_insert(etab, eh - 1, pair_l[p], &overflow);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < eh; s += blockDim.x) {
    int32_t l = etab[s];
    if (l < 0) continue;
    for (int c = 0; c < nb; c++)
      if (hash_insert(ntab, nh - 1, conn[(int64_t)l * nb + c], &overflow)) atomicAdd(&ncount, 1);
  }
  __syncthreads();
  if (overflow || ncount * 4 > nh * 3) {
    if (threadIdx.x == 0) atomicOr(err, ERR_HASH_FULL);
    return;
  }
  if (MODE != 1) {
    if (threadIdx.x == 0) {
      row_cnt[i] = ncount;
      atomicMax(max_row, ncount);
    }
    if (MODE == 0) return;
  }
  int n = ncount;
  if (MODE == 1 && (int64_t)n != row_ptr[i + 1] - row_ptr[i]) {
    if (threadIdx.x == 0) atomicOr(err, ERR_ROW_COUNT);
    return;
  }
  if (MODE == 2 && n > rowcap) {
    if (threadIdx.x == 0) atomicOr(err, ERR_HASH_FULL);
    return;
  }
  // compact the node set into etab[0..n), then sort
  __shared__ int cpos;
  if (threadIdx.x == 0) cpos = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nh; s += blockDim.x) {
    int32_t v = ntab[s];
    if (v >= 0) etab[atomicAdd(&cpos, 1)] = v;
  }
  __syncthreads();
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int t = n + threadIdx.x; t < np2; t += blockDim.x) etab[t] = INT_MAX;
  __syncthreads();
  block_bitonic_sort(etab, np2);
  if (MODE == 1) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) col[row_ptr[i] + t] = etab[t];
  } else {
    for (int t = threadIdx.x; t < n; t += blockDim.x) tmp[i * (int64_t)rowcap + t] = etab[t];
  }
}

// Packs the staged sorted rows (k_rows MODE 2) into the CSR column array (warp per row).
__global__ void k_copy_rows(int64_t n_vert, int rowcap, const int32_t* __restrict__ tmp,
                            const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n_vert) return;
  const int64_t b = row_ptr[i], n = row_ptr[i + 1] - b;
  for (int64_t t = lane; t < n; t += 32) col[b + t] = tmp[i * (int64_t)rowcap + t];
}

int next_pow2(int64_t v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

void pairs_release(nl_pairs* p) {
  if (!p) return;
  if (p->refs.fetch_sub(1) != 1) return;
  cudaStream_t s = p->mesh ? p->mesh->stream : nullptr;
  dev_free(p->pair_off, 0, s);
  dev_free(p->pair_l, 0, s);
  dev_free(p->row_ptr, 0, s);
  dev_free(p->col, 0, s);
  cudaStreamSynchronize(s);
  mesh_release(p->mesh);
  delete p;
}

template <int D>
static nl_status build_pairs_dim(nl_mesh* m, double delta, double eps, nl_pairs* out) {
  cudaStream_t s = m->stream;
  const double reach = delta + eps;
  const int64_t ne = m->n_elem, nvv = m->n_vert;
  // grid
  Grid g;
  double side = (reach + m->max_ext) * (1.0 + 1e-9);
  int64_t total = 1;
  for (int k = 0; k < 3; k++) {
    g.lo[k] = m->bb_lo[k];
    g.n[k] = 1;
  }
  for (int k = 0; k < D; k++) {
    double ext = m->bb_hi[k] - m->bb_lo[k];
    g.n[k] = (int)std::max(1.0, std::ceil(ext / side));
  }
  for (int k = 0; k < D; k++) total *= g.n[k];
  while (total > (1 << 24)) {  // keep the cell table small: larger cells stay correct
    side *= 2.0;
    total = 1;
    for (int k = 0; k < D; k++) {
      g.n[k] = (int)std::max(1.0, std::ceil((m->bb_hi[k] - m->bb_lo[k]) / side));
      total *= g.n[k];
    }
  }
  g.inv_s = 1.0 / side;
  // re-check the neighbour property against the rounded reciprocal: cells of side 1/inv_s
  if (1.0 / g.inv_s < reach + m->max_ext) g.inv_s = 1.0 / ((reach + m->max_ext) * (1.0 + 1e-6));

  DevBuf<int32_t> cell_cnt, cursor, items, max_cnt, err;
  DevBuf<int64_t> cell_off, cnt;
  NL_TRY(cell_cnt.alloc(total, s));
  NL_TRY(cursor.alloc(total, s));
  NL_TRY(cell_off.alloc(total + 1, s));
  NL_TRY(items.alloc(ne, s));
  NL_TRY(cnt.alloc(ne, s));
  NL_TRY(max_cnt.alloc(2, s));
  NL_TRY(err.alloc(1, s));
  NL_CUDA(cudaMemsetAsync(cell_cnt.p, 0, sizeof(int32_t) * total, s));
  NL_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * total, s));
  NL_CUDA(cudaMemsetAsync(max_cnt.p, 0, sizeof(int32_t) * 2, s));
  NL_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int32_t), s));
  const int tb = 256;
  unsigned gb = (unsigned)((ne + tb - 1) / tb);
  // FP32 boxes for the screened test; margin: 8 FP32 ulps of the largest coordinate magnitude
  // plus the reach, far above the rounding of the boxes (1 ulp each) and of the subtraction
  DevBuf<float> fbox;
  NL_TRY(fbox.alloc((size_t)2 * D * ne, s));
  {
    const int64_t nn = (int64_t)D * ne;
    k_round_boxes<<<NL_CNT((unsigned)((nn + tb - 1) / tb)), tb, 0, s>>>(nn, m->blo, m->bhi, fbox.p,
                                                                       fbox.p + nn);
  }
  double cmax = 0.0;
  for (int k = 0; k < D; k++) cmax = std::max(cmax, std::max(std::fabs(m->bb_lo[k]), std::fabs(m->bb_hi[k])));
  const double margin = 8.0 * 1.1920928955078125e-07 * (cmax + reach);
  Screen S{fbox.p, fbox.p + (size_t)D * ne, (float)(reach - margin), (float)(reach + margin)};
  k_bin_count<D><<<NL_CNT(gb), tb, 0, s>>>(ne, g, m->blo, m->bhi, cell_cnt.p);
  NL_TRY(exclusive_scan_i32_to_i64(cell_cnt.p, cell_off.p, total, s));
  k_bin_fill<D><<<NL_CNT(gb), tb, 0, s>>>(ne, g, m->blo, m->bhi, cell_off.p, cursor.p, items.p);
  unsigned gw = (unsigned)((ne * 32 + tb - 1) / tb);
  k_pairs_count<D><<<NL_CNT(gw), tb, 0, s>>>(ne, g, reach, m->blo, m->bhi, cell_off.p, items.p, cnt.p,
                                     max_cnt.p, S);
  NL_CUDA(cudaGetLastError());
  DevBuf<int64_t> off;
  NL_TRY(off.alloc(ne + 1, s));
  NL_TRY(exclusive_scan_i64(cnt.p, off.p, ne, s));
  int64_t n_pairs = 0;
  int32_t mx = 0;
  NL_CUDA(cudaMemcpyAsync(&n_pairs, off.p + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaMemcpyAsync(&mx, max_cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  const int cap_limit = 49152;
  if (mx > cap_limit)
    return fail(NL_EINTERNAL, "nl_pairs_build: %d pairs for one element exceed the capacity %d",
                mx, cap_limit);
  DevBuf<int32_t> pl;
  NL_TRY(pl.alloc(n_pairs > 0 ? n_pairs : 1, s));
  int cap = next_pow2(std::max<int64_t>(mx, 1));
  size_t smem = sizeof(int32_t) * cap;
  NL_TRY(allow_smem(k_pairs_fill<D>, smem));
  k_pairs_fill<D><<<NL_CNT((unsigned)ne), 256, smem, s>>>(ne, g, reach, m->blo, m->bhi, cell_off.p, items.p,
                                                 off.p, pl.p, cap, err.p, S);
  NL_CUDA(cudaGetLastError());

  // pattern
  DevBuf<int64_t> maxs;
  NL_TRY(maxs.alloc(1, s));
  NL_CUDA(cudaMemsetAsync(maxs.p, 0, sizeof(int64_t), s));
  k_row_bound<<<NL_CNT((unsigned)((nvv + tb - 1) / tb)), tb, 0, s>>>(nvv, m->n2e_off, m->n2e, off.p, maxs.p);
  int64_t max_sum = 0;
  NL_CUDA(cudaMemcpyAsync(&max_sum, maxs.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  int eh = next_pow2(std::max<int64_t>(64, std::min<int64_t>(2 * max_sum, 32768)));
  // node table: a P2 (or quadrilateral) element brings about four (two) times the nodes of a
  // P1 triangle into a row, a Q2 or serendipity hexahedron up to eight times those of a Q1
  // one; the element table is at least as large, as the sorted row is staged in it
  int nh = std::min(8192, (m->cell == 2 && m->order >= 2) ? 8 * eh
                          : (m->order == 2 || m->cell == 1) ? 2 * eh : eh);
  eh = std::max(eh, nh);
  size_t rsmem = sizeof(int32_t) * (eh + nh);
  NL_TRY((allow_smem(k_rows<D, 0>, rsmem)));
  NL_TRY((allow_smem(k_rows<D, 1>, rsmem)));
  NL_TRY((allow_smem(k_rows<D, 2>, rsmem)));
  DevBuf<int32_t> rcnt;
  NL_TRY(rcnt.alloc(nvv, s));
  // one pass that counts and sorts each row into a staging area of rowcap columns per row (the
  // row's capacity check keeps every row below 3/4 of the node table), when that area fits in
  // a quarter of the free memory (and 4 GiB); otherwise a counting pass and a filling pass
  const int rowcap = nh * 3 / 4;
  size_t free_b = 0, total_b = 0;
  NL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t stage_bytes = (size_t)nvv * (size_t)rowcap * sizeof(int32_t);
  const bool staged = stage_bytes <= std::min<size_t>(free_b / 4, (size_t)4 << 30);
  DevBuf<int32_t> stage;
  if (staged) {
    NL_TRY(stage.alloc(stage_bytes / sizeof(int32_t), s));
    k_rows<D, 2><<<NL_CNT((unsigned)nvv), 256, rsmem, s>>>(nvv, m->conn, m->nb, m->n2e_off, m->n2e, off.p, pl.p,
                                                       eh, nh, rcnt.p, nullptr, nullptr, err.p,
                                                       max_cnt.p + 1, stage.p, rowcap);
  } else {
    k_rows<D, 0><<<NL_CNT((unsigned)nvv), 256, rsmem, s>>>(nvv, m->conn, m->nb, m->n2e_off, m->n2e, off.p, pl.p,
                                                       eh, nh, rcnt.p, nullptr, nullptr, err.p,
                                                       max_cnt.p + 1, nullptr, 0);
  }
  NL_CUDA(cudaGetLastError());
  DevBuf<int64_t> rp;
  NL_TRY(rp.alloc(nvv + 1, s));
  NL_TRY(exclusive_scan_i32_to_i64(rcnt.p, rp.p, nvv, s));
  int64_t nnz = 0;
  int e = 0, max_row = 0;
  NL_CUDA(cudaMemcpyAsync(&nnz, rp.p + nvv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaMemcpyAsync(&max_row, max_cnt.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  if (e) {
    return fail(NL_EINTERNAL, "nl_pairs_build: device check failed (code %d%s)", e,
                (e & ERR_HASH_FULL) ? ": a row neighbourhood exceeds the shared-memory hash capacity"
                                    : "");
  }
  DevBuf<int32_t> col;
  NL_TRY(col.alloc(nnz > 0 ? nnz : 1, s));
  if (staged) {
    k_copy_rows<<<NL_CNT((unsigned)((nvv * 32 + 255) / 256)), 256, 0, s>>>(nvv, rowcap, stage.p, rp.p, col.p);
  } else {
    k_rows<D, 1><<<NL_CNT((unsigned)nvv), 256, rsmem, s>>>(nvv, m->conn, m->nb, m->n2e_off, m->n2e, off.p, pl.p,
                                                       eh, nh, nullptr, rp.p, col.p, err.p, nullptr,
                                                       nullptr, 0);
  }
  NL_CUDA(cudaGetLastError());
  NL_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  if (e) return fail(NL_EINTERNAL, "nl_pairs_build: device check failed in the fill pass (code %d)", e);
  out->n_pairs = n_pairs;
  out->nnz = nnz;
  out->max_pairs_per_elem = mx;
  out->max_row_nnz = max_row;
  out->pair_off = off.release_ownership();
  out->pair_l = pl.release_ownership();
  out->row_ptr = rp.release_ownership();
  out->col = col.release_ownership();
  return NL_OK;
}

nl_status build_pairs(nl_mesh* m, double delta, double eps, nl_pairs* out) {
  out->mesh = m;
  m->refs.fetch_add(1);
  out->delta = delta;
  out->eps = eps;
  return m->dim == 2 ? build_pairs_dim<2>(m, delta, eps, out) : build_pairs_dim<3>(m, delta, eps, out);
}

}  // namespace nlx
