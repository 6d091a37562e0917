// AMR cycle on the device (Sec. 7: the AMR callback every N_AMR steps; Sec. 6.2: the level
// partition re-assigned after it).
//
// The leaves of every ensemble member are kept in Morton order (member-major), which the
// adaptation preserves in place: a refined leaf is replaced by its four children in Morton
// order, four coarsened siblings (consecutive in Morton order) by their parent at the first
// sibling's position.  The whole plan therefore runs on the device:
//   k_amr_desired    indicator -> desired level (refine above / coarsen below thresholds)
//   k_amr_balance    least fixed point of the sibling rule and the 2:1 face rule (one block,
//                    monotone raising until a pass changes nothing)
//   k_amr_scan       output count of every old leaf (4, 1 or 0), exclusive scan, new size
//   k_amr_leaves     new leaves, their Morton keys and the transfer records
//   k_connect<W>     interfaces and mortars of the new leaves, found by binary search of face
//                    neighbour points among the sorted Morton keys; counted, scanned
//                    (k_scan_faces), then written in the order the host builder uses (element
//                    by element; per direction the +dir record, then the -dir mortar)
//   k_amr_install    levels and members of the new leaves
// after which the transfer kernel moves the solution and the partition kernel rebuilds the
// sorted lists.  Every decision is an integer one, so the result is the host plan's, bit for bit.

#include <cuda_runtime.h>
#include <stdint.h>

#include "perk.h"
#include "perk_internal.h"

namespace perk {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int KEY_LEVEL = 20;   // Morton keys at the resolution of level 20 (the deepest level)

// spreads the low 20 bits of x to the even bit positions
__device__ __forceinline__ unsigned long long spread(unsigned long long x) {
  x &= 0xFFFFFull;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

// (member, Morton key of the cell's lower-left corner at level 20): sorts member-major, Morton within
__device__ __forceinline__ unsigned long long cell_key(int member, int l, int ix, int iy) {
  const unsigned long long X = (unsigned long long)ix << (KEY_LEVEL - l);
  const unsigned long long Y = (unsigned long long)iy << (KEY_LEVEL - l);
  return ((unsigned long long)member << 40) | spread(X) | (spread(Y) << 1);
}

// index of the leaf containing the lower-left corner of cell (l, ix, iy) of `member`: the last
// leaf whose key does not exceed the corner's (the leaves' Morton intervals tile each member)
__device__ __forceinline__ int find_leaf(const unsigned long long* __restrict__ key, int n, int member, int l, int ix,
                                         int iy) {
  const unsigned long long k = cell_key(member, l, ix, iy);
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key[mid] <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// block-wide exclusive scan of one value per thread (SCAN_THREADS threads); returns the
// exclusive prefix and writes the block total to *total
__device__ int block_exclusive_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = s_warp[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const int r = s_warp[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void k_amr_desired(int64_t n, const double* __restrict__ eta, const int4* __restrict__ cells, int lmin,
                              int lmax, double refine_above, double coarsen_below, int32_t* __restrict__ d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int l = cells[e].x;
  const double v = eta[e];
  int t = l;
  if (v > refine_above && l < lmax)
    t = l + 1;
  else if (v < coarsen_below && l > lmin && !(v > refine_above))
    t = l - 1;
  d[e] = t;
}

// whether leaf e (level l > 0) has its three siblings as leaves (consecutive in Morton order) and
// all four want to coarsen
__device__ __forceinline__ bool group_coarsens(int64_t n, const int4* __restrict__ cells, const int32_t* d, int64_t e,
                                               int4 c) {
  const int child = (c.y & 1) | ((c.z & 1) << 1);
  const int64_t k = e - child;
  if (k < 0 || k + 3 >= n) return false;
  for (int j = 0; j < 4; ++j) {
    const int4 s = cells[k + j];
    if (s.x != c.x || s.w != c.w || (s.y >> 1) != (c.y >> 1) || (s.z >> 1) != (c.z >> 1) ||
        ((s.y & 1) | ((s.z & 1) << 1)) != j)
      return false;
    if (!(((volatile const int32_t*)d)[k + j] < s.x)) return false;
  }
  return true;
}

// Least fixed point >= d of: a leaf coarsens only with its three siblings (all leaves, all wanting
// to), and face neighbours of the new mesh differ by at most one level.  Values only rise, each
// rise to the least value the violated rule needs given values that are themselves below the
// least fixed point, so the first pass without a change ends at that fixed point whatever the
// order of the updates.
// Every pass that changes something raises some value by at least one, and no value exceeds the
// largest level + 1, so the loop ends; MAX_BALANCE_PASSES only guards that bound (info[4] = 1).
constexpr int MAX_BALANCE_PASSES = 4096;

__global__ void __launch_bounds__(SCAN_THREADS) k_amr_balance(int64_t n, const int4* __restrict__ cells, int64_t n_if,
                                                              const int4* __restrict__ ifs, int64_t n_mort,
                                                              const int4* __restrict__ morts, int32_t* d,
                                                              int64_t* info) {
  __shared__ int s_changed;
  if (threadIdx.x == 0) info[4] = 0;
  for (int pass = 0;; ++pass) {
    if (pass == MAX_BALANCE_PASSES) {
      if (threadIdx.x == 0) info[4] = 1;
      break;
    }
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();
    int changed = 0;
    for (int64_t e = threadIdx.x; e < n; e += SCAN_THREADS) {
      const int4 c = cells[e];
      if (d[e] < c.x && (c.x == 0 || !group_coarsens(n, cells, d, e, c))) {
        atomicMax(&d[e], c.x);
        changed = 1;
      }
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < n_if + 2 * n_mort; q += SCAN_THREADS) {
      int a, b;
      if (q < n_if) {
        a = ifs[q].x;
        b = ifs[q].y;
      } else {
        const int4 m = morts[(q - n_if) >> 1];
        a = m.x;
        b = ((q - n_if) & 1) ? m.z : m.y;
      }
      const int da = ((volatile int32_t*)d)[a], db = ((volatile int32_t*)d)[b];
      if (da > db + 1) {
        atomicMax(&d[b], da - 1);
        changed = 1;
      } else if (db > da + 1) {
        atomicMax(&d[a], db - 1);
        changed = 1;
      }
    }
    if (changed) s_changed = 1;
    __syncthreads();
    const int any = s_changed;
    __syncthreads();
    if (!any) break;
  }
}

// per old leaf the number of new leaves it yields (4 refined, 1 kept, 1 for the first of four
// coarsened siblings, 0 for the others); exclusive offsets, the new count and a change flag
__global__ void __launch_bounds__(SCAN_THREADS) k_amr_scan(int64_t n, const int4* __restrict__ cells,
                                                           const int32_t* __restrict__ d, int32_t* __restrict__ off,
                                                           int64_t* info) {
  __shared__ int s_warp[32];
  __shared__ int s_total;
  int64_t carry = 0;
  int changed = 0;
  for (int64_t start = 0; start < n; start += SCAN_THREADS) {
    const int64_t e = start + threadIdx.x;
    int cnt = 0;
    if (e < n) {
      const int4 c = cells[e];
      const int t = d[e];
      if (t != c.x) changed = 1;
      cnt = t > c.x ? 4 : t == c.x ? 1 : (((c.y & 1) | (c.z & 1)) == 0 ? 1 : 0);
    }
    const int ex = block_exclusive_scan(cnt, s_warp, &s_total);
    if (e < n) off[e] = (int32_t)(carry + ex);
    carry += s_total;
    __syncthreads();
  }
  changed = __syncthreads_or(changed);
  if (threadIdx.x == 0) {
    off[n] = (int32_t)carry;
    info[0] = carry;
    info[1] = changed;
  }
}

// new leaves (level, ix, iy, member), their keys, and the transfer records of k_transfer:
// rec[0] = kind | cx << 2 | cy << 3 (0 copy, 1 child of a refined cell, 2 parent of four), rec[1..4]
// the old source leaves (children in Morton order)
__global__ void k_amr_leaves(int64_t n, const int4* __restrict__ cells, const int32_t* __restrict__ d,
                             const int32_t* __restrict__ off, int4* __restrict__ out, unsigned long long* __restrict__ key,
                             int32_t* __restrict__ map) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int4 c = cells[e];
  const int t = d[e];
  const int64_t o = off[e];
  if (t > c.x) {
    for (int ch = 0; ch < 4; ++ch) {
      const int cx = ch & 1, cy = ch >> 1;
      const int4 q = make_int4(c.x + 1, 2 * c.y + cx, 2 * c.z + cy, c.w);
      out[o + ch] = q;
      key[o + ch] = cell_key(q.w, q.x, q.y, q.z);
      int32_t* r = map + 5 * (o + ch);
      r[0] = 1 | (cx << 2) | (cy << 3);
      r[1] = (int32_t)e;
      r[2] = r[3] = r[4] = 0;
    }
  } else if (t == c.x) {
    out[o] = c;
    key[o] = cell_key(c.w, c.x, c.y, c.z);
    int32_t* r = map + 5 * o;
    r[0] = 0;
    r[1] = (int32_t)e;
    r[2] = r[3] = r[4] = 0;
  } else if (((c.y & 1) | (c.z & 1)) == 0) {
    const int4 q = make_int4(c.x - 1, c.y >> 1, c.z >> 1, c.w);
    out[o] = q;
    key[o] = cell_key(q.w, q.x, q.y, q.z);
    int32_t* r = map + 5 * o;
    r[0] = 2;
    for (int j = 0; j < 4; ++j) r[1 + j] = (int32_t)(e + j);
  }
}

// Face couplings of leaf e of a periodic, 2:1-balanced leaf list in key order.  For each
// direction: the +dir neighbour region of the same size is a leaf (interface e -> it), lies in a
// coarser leaf (e is the small side of a mortar built from the other side), or is refined (mortar
// with e as the large side, large_side 0); the -dir region only yields the mortars with e as the
// large side (large_side 1).  COUNT: cnt_if[e], cnt_mort[e]; WRITE: records at off_*[e].
template <bool WRITE>
__global__ void k_connect(int64_t n, const int4* __restrict__ cells, const unsigned long long* __restrict__ key,
                          int32_t* __restrict__ cnt_if, int32_t* __restrict__ cnt_mort,
                          const int32_t* __restrict__ off_if, const int32_t* __restrict__ off_mort,
                          int4* __restrict__ ifs, int4* __restrict__ morts) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int4 c = cells[e];
  const int l = c.x, m = c.w, side = 1 << l, nn = (int)n;
  int ni = 0, nm = 0;
  const int64_t oi = WRITE ? off_if[e] : 0, om = WRITE ? off_mort[e] : 0;
  for (int dir = 0; dir < 2; ++dir) {
    {
      const int px = dir == 0 ? (c.y + 1) & (side - 1) : c.y;
      const int py = dir == 1 ? (c.z + 1) & (side - 1) : c.z;
      const int f = find_leaf(key, nn, m, l, px, py);
      const int lf = cells[f].x;
      if (lf == l) {
        if (WRITE) ifs[oi + ni] = make_int4((int)e, f, dir, 0);
        ++ni;
      } else if (lf == l + 1) {
        const int cx0 = 2 * px, cy0 = 2 * py;
        const int s1 = find_leaf(key, nn, m, l + 1, dir == 0 ? cx0 : cx0 + 1, dir == 0 ? cy0 + 1 : cy0);
        if (WRITE) morts[om + nm] = make_int4((int)e, f, s1, dir | (0 << 1));
        ++nm;
      }
    }
    {
      // the -dir region's half-size cell touching e's face (its corner cell does not touch the
      // face and may be finer): a leaf of level l + 1 there means the region is refined
      const int mx = dir == 0 ? (c.y + side - 1) & (side - 1) : c.y;
      const int my = dir == 1 ? (c.z + side - 1) & (side - 1) : c.z;
      const int cx0 = dir == 0 ? 2 * mx + 1 : 2 * mx, cy0 = dir == 0 ? 2 * my : 2 * my + 1;
      const int s0 = l < KEY_LEVEL ? find_leaf(key, nn, m, l + 1, cx0, cy0) : -1;
      if (s0 >= 0 && cells[s0].x == l + 1) {
        const int s1 = find_leaf(key, nn, m, l + 1, dir == 0 ? cx0 : cx0 + 1, dir == 0 ? cy0 + 1 : cy0);
        if (WRITE) morts[om + nm] = make_int4((int)e, s0, s1, dir | (1 << 1));
        ++nm;
      }
    }
  }
  if (!WRITE) {
    cnt_if[e] = ni;
    cnt_mort[e] = nm;
  }
}

// exclusive scans of the per-leaf interface and mortar counts; totals to info[2], info[3]
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_faces(int64_t n, const int32_t* __restrict__ cnt_if,
                                                             const int32_t* __restrict__ cnt_mort,
                                                             int32_t* __restrict__ off_if, int32_t* __restrict__ off_mort,
                                                             int64_t* info) {
  __shared__ int s_warp[32];
  __shared__ int s_total;
  int64_t ci = 0, cm = 0;
  for (int64_t start = 0; start < n; start += SCAN_THREADS) {
    const int64_t e = start + threadIdx.x;
    const int vi = e < n ? cnt_if[e] : 0, vm = e < n ? cnt_mort[e] : 0;
    const int xi = block_exclusive_scan(vi, s_warp, &s_total);
    const int64_t ti = s_total;
    const int xm = block_exclusive_scan(vm, s_warp, &s_total);
    const int64_t tm = s_total;
    if (e < n) {
      off_if[e] = (int32_t)(ci + xi);
      off_mort[e] = (int32_t)(cm + xm);
    }
    ci += ti;
    cm += tm;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    info[2] = ci;
    info[3] = cm;
  }
}

__global__ void k_amr_install(int64_t n, const int4* __restrict__ cells, int32_t* __restrict__ level,
                              int32_t* __restrict__ member) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int4 c = cells[e];
  level[e] = c.x;
  member[e] = c.w;
}

inline unsigned grid_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_amr_plan(cudaStream_t st, int64_t n, const int4* cells, const double* eta, const AmrPlanArgs& a,
                            int64_t n_if, const int4* ifs, int64_t n_mort, const int4* morts, int32_t* d,
                            int32_t* off, int64_t* info) {
  if (n <= 0) return cudaErrorInvalidValue;
  if (eta) {
    k_amr_desired<<<grid_of(n, 256), 256, 0, st>>>(n, eta, cells, a.level_min, a.level_max, a.refine_above,
                                                   a.coarsen_below, d);
  }
  k_amr_balance<<<1, SCAN_THREADS, 0, st>>>(n, cells, n_if, ifs, n_mort, morts, d, info);
  k_amr_scan<<<1, SCAN_THREADS, 0, st>>>(n, cells, d, off, info);
  return cudaGetLastError();
}

cudaError_t launch_amr_leaves(cudaStream_t st, int64_t n, const int4* cells, const int32_t* d, const int32_t* off,
                              int4* out, unsigned long long* key, int32_t* map) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_amr_leaves<<<grid_of(n, 256), 256, 0, st>>>(n, cells, d, off, out, key, map);
  return cudaGetLastError();
}

cudaError_t launch_connect(cudaStream_t st, int64_t n, const int4* cells, const unsigned long long* key,
                           int32_t* cnt_if, int32_t* cnt_mort, int32_t* off_if, int32_t* off_mort, int4* ifs,
                           int4* morts, int64_t* info) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_connect<false><<<grid_of(n, 128), 128, 0, st>>>(n, cells, key, cnt_if, cnt_mort, nullptr, nullptr, nullptr,
                                                    nullptr);
  k_scan_faces<<<1, SCAN_THREADS, 0, st>>>(n, cnt_if, cnt_mort, off_if, off_mort, info);
  k_connect<true><<<grid_of(n, 128), 128, 0, st>>>(n, cells, key, nullptr, nullptr, off_if, off_mort, ifs, morts);
  return cudaGetLastError();
}

cudaError_t launch_amr_install(cudaStream_t st, int64_t n, const int4* cells, int32_t* level, int32_t* member) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_amr_install<<<grid_of(n, 256), 256, 0, st>>>(n, cells, level, member);
  return cudaGetLastError();
}

}  // namespace perk
