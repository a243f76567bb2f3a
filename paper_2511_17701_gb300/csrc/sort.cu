// sort.cu -- stable counting sort of a species by tile-major cell key (an addition of
// this library: the paper's loop does not sort). Least-significant-digit radix passes
// of 8 bits; each pass is upsweep (per-block digit histogram), an exclusive scan of the
// digit-major histogram, and a downsweep where each warp ranks its own contiguous run
// with __match_any_sync, so the order of equal keys is the input order and the
// permutation is unique (bit-exact). Particles not alive get the key 0xFFFFFFFF, sort
// last and are dropped.
#include "grpic_internal.cuh"

namespace {

constexpr int TPB = 256;                      // 8 warps
constexpr int NWARP = TPB / 32;
constexpr int ITEMS = 16;                     // per lane and pass
constexpr int WCHUNK = 32 * ITEMS;            // contiguous elements per warp
constexpr int BCHUNK = NWARP * WCHUNK;        // contiguous elements per block
constexpr int SCAN_SEG = 1024;

__device__ __forceinline__ uint32_t cell_key(int i1, int i2, uint8_t tag, int n_r, int tr, int tt) {
  if (tag != 1) return 0xFFFFFFFFu;
  const uint32_t ntr = (uint32_t)((n_r + tr - 1) / tr);
  const uint32_t tile = (uint32_t)(i2 / tt) * ntr + (uint32_t)(i1 / tr);
  return tile * (uint32_t)(tr * tt) + (uint32_t)(i2 % tt) * (uint32_t)tr + (uint32_t)(i1 % tr);
}

// keys and the identity permutation; the live count is summed per thread, reduced within
// the block and added with one atomic per block (one per warp and iteration serialised on
// the single counter: 0.23 ms per 8.4 M particles)
template <typename T>
__global__ void __launch_bounds__(TPB) k_keys(SpeciesDevT<T> s, int n_r, int tr, int tt,
                                              uint32_t *keys, uint32_t *vals,
                                              unsigned long long *alive) {
  __shared__ unsigned wsum[NWARP];
  constexpr int U = 4;  // elements per thread and trip, loaded before any is stored
  const int64_t n = *s.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned cnt = 0;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < n; k0 += U * stride) {
    int a1[U], a2[U];
    uint8_t tg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = k0 + u * stride;
      if (k < n) {
        tg[u] = s.tag[k];
        a1[u] = s.i1[k];
        a2[u] = s.i2[k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = k0 + u * stride;
      if (k < n) {
        keys[k] = cell_key(a1[u], a2[u], tg[u], n_r, tr, tt);
        vals[k] = (uint32_t)k;
        cnt += tg[u] == 1 ? 1u : 0u;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < NWARP; ++w) t += wsum[w];
    if (t) atomicAdd(alive, t);
  }
}

// After the sort: tile_start[t] = the first particle of tile t (keys ascending, the dropped
// particles last), t = 0 .. n_tiles; tile_start[n_tiles] = the live count.
__global__ void k_tile_ranges(const uint32_t *keys, const int64_t *n_dev, int n_tiles,
                              uint32_t cells_per_tile, uint32_t *tile_start) {
  const int64_t n = *n_dev;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= n_tiles; t += gridDim.x * blockDim.x) {
    const uint64_t target = (uint64_t)t * cells_per_tile;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((uint64_t)keys[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    tile_start[t] = (uint32_t)lo;
  }
}

__global__ void k_hist(const uint32_t *keys, const int64_t *n_dev, int shift, int nblocks,
                       uint32_t *hist) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t n = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * BCHUNK;
  const int64_t end = min(n, base + BCHUNK);
  for (int64_t e = base + threadIdx.x; e < end; e += TPB)
    atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_scatter(const uint32_t *kin, const uint32_t *vin, uint32_t *kout,
                          uint32_t *vout, const int64_t *n_dev, int shift, int nblocks,
                          const uint32_t *offs) {
  __shared__ uint32_t wcnt[NWARP][256];
  __shared__ uint32_t wbase[NWARP][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < NWARP * 256; d += TPB) (&wcnt[0][0])[d] = 0;
  __syncthreads();
  const int64_t n = *n_dev;
  const int64_t wb = (int64_t)blockIdx.x * BCHUNK + (int64_t)w * WCHUNK;
  for (int b = 0; b < ITEMS; ++b) {
    const int64_t e = wb + b * 32 + lane;
    if (e < n) atomicAdd(&wcnt[w][(kin[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  {
    const int d = threadIdx.x;  // TPB == 256 digits
    uint32_t run = offs[(int64_t)d * nblocks + blockIdx.x];
    for (int v = 0; v < NWARP; ++v) {
      wbase[v][d] = run;
      run += wcnt[v][d];
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int b = 0; b < ITEMS; ++b) {
    const int64_t e = wb + b * 32 + lane;
    const bool ok = e < n;
    const uint32_t key = ok ? kin[e] : 0u;
    const uint32_t d = ok ? ((key >> shift) & 255u) : (256u + lane);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    uint32_t pos = 0;
    if (ok) pos = wbase[w][d] + __popc(peers & lt);
    __syncwarp();
    if (ok) {
      kout[pos] = key;
      vout[pos] = vin[e];
      if (lane == __ffs(peers) - 1) wbase[w][d] += __popc(peers);
    }
    __syncwarp();
  }
}

// Exclusive scan of one value per thread across the block (blockDim.x a multiple of 32, at
// most 1024): warp shuffles, then the warp totals scanned by the first warp. Returns the
// thread's exclusive prefix and sets *total to the block's sum. Every thread calls it; the
// shared array is reused, so calls are separated by a barrier.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ uint32_t ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < nw ? ws[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, t, d);
      if (lane >= d) t += y;
    }
    ws[lane] = t;  // inclusive prefix of the warp totals
  }
  __syncthreads();
  *total = ws[nw - 1];
  return (w ? ws[w - 1] : 0u) + x - v;
}

// exclusive scan of a uint32 array in segments of SCAN_SEG (blocks of SCAN_SEG / 4 threads,
// four consecutive elements each), segment totals to bsum
__global__ void __launch_bounds__(SCAN_SEG / 4) k_scan_seg(uint32_t *a, int64_t L,
                                                           uint32_t *bsum) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_SEG + 4 * threadIdx.x;
  uint32_t v[4], sum = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < L ? a[base + j] : 0u;
    sum += v[j];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(sum, &total);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < L) a[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// exclusive scan of the S segment totals: one block, 4 consecutive entries per thread and
// chunk, a running carry across chunks
constexpr int SCAN_SUMS_TPB = 1024;
__global__ void __launch_bounds__(SCAN_SUMS_TPB) k_scan_sums(uint32_t *bsum, int64_t S) {
  uint32_t carry = 0;
  for (int64_t c0 = 0; c0 < S; c0 += 4 * (int64_t)blockDim.x) {
    const int64_t base = c0 + 4 * threadIdx.x;
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = base + j < S ? bsum[base + j] : 0u;
      sum += v[j];
    }
    uint32_t total;
    uint32_t run = carry + block_exclusive_scan(sum, &total);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (base + j < S) bsum[base + j] = run;
      run += v[j];
    }
    carry += total;
    __syncthreads();  // the scan's shared array is read above before the next chunk writes it
  }
}

__global__ void k_scan_add(uint32_t *a, int64_t L, const uint32_t *bsum) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < L) a[t] += bsum[t / SCAN_SEG];
}

// gather every array of the species by the final permutation (PREV false: all but the
// previous position). Each thread takes GATHER_U elements a grid stride apart and issues all
// their loads before any store, so that enough reads are in flight to cover the latency of
// the permuted loads that depend on perm.
constexpr int GATHER_U = 4;
template <typename T, bool PREV>
__global__ void __launch_bounds__(TPB) k_gather(SpeciesDevT<T> in, SpeciesDevT<T> out,
                                                const uint32_t *__restrict__ perm,
                                                const int64_t *n_dev) {
  const int64_t n = *n_dev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < n;
       k0 += GATHER_U * stride) {
    uint32_t p[GATHER_U];
    bool ok[GATHER_U];
#pragma unroll
    for (int u = 0; u < GATHER_U; ++u) {
      ok[u] = k0 + u * stride < n;
      p[u] = ok[u] ? __ldg(perm + k0 + u * stride) : 0u;
    }
    int32_t i1[GATHER_U], i2[GATHER_U], i1p[GATHER_U], i2p[GATHER_U];
    T dx1[GATHER_U], dx2[GATHER_U], u1[GATHER_U], u2[GATHER_U], u3[GATHER_U], phi[GATHER_U],
        w[GATHER_U], dx1p[GATHER_U], dx2p[GATHER_U];
    uint8_t tag[GATHER_U];
#pragma unroll
    for (int u = 0; u < GATHER_U; ++u) {
      if (!ok[u]) continue;
      const uint32_t q = p[u];
      i1[u] = in.i1[q]; i2[u] = in.i2[q];
      dx1[u] = in.dx1[q]; dx2[u] = in.dx2[q];
      u1[u] = in.u1[q]; u2[u] = in.u2[q]; u3[u] = in.u3[q];
      phi[u] = in.phi[q]; w[u] = in.w[q]; tag[u] = in.tag[q];
      if (PREV) {
        i1p[u] = in.i1p[q]; i2p[u] = in.i2p[q];
        dx1p[u] = in.dx1p[q]; dx2p[u] = in.dx2p[q];
      }
    }
#pragma unroll
    for (int u = 0; u < GATHER_U; ++u) {
      if (!ok[u]) continue;
      const int64_t k = k0 + u * stride;
      out.i1[k] = i1[u]; out.i2[k] = i2[u];
      out.dx1[k] = dx1[u]; out.dx2[k] = dx2[u];
      out.u1[k] = u1[u]; out.u2[k] = u2[u]; out.u3[k] = u3[u];
      out.phi[k] = phi[u]; out.w[k] = w[u]; out.tag[k] = tag[u];
      if (PREV) {
        out.i1p[k] = i1p[u]; out.i2p[k] = i2p[u];
        out.dx1p[k] = dx1p[u]; out.dx2p[k] = dx2p[u];
      }
    }
  }
}

__global__ void k_set_n(int64_t *n_dev, const unsigned long long *alive) {
  *n_dev = (int64_t)*alive;
}

int grid_for(int64_t n, int tpb) {
  int64_t b = (n + tpb - 1) / tpb;
  if (b > 152 * 64) b = 152 * 64;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int64_t sort_hist_entries(int64_t max_n) {
  const int64_t nb = (max_n + BCHUNK - 1) / BCHUNK;
  return 256 * (nb < 1 ? 1 : nb);
}
int64_t sort_bsum_entries(int64_t max_n) {
  return (sort_hist_entries(max_n) + SCAN_SEG - 1) / SCAN_SEG;
}

template <typename T>
cudaError_t launch_sort(const GridP &g, int tr, int tt, SpeciesDevT<T> in, SpeciesDevT<T> out,
                        int64_t n_bound, int64_t *n_dev, const SortScratch &S,
                        uint32_t *tile_start, cudaStream_t st, bool with_prev) {
  if (n_bound <= 0) return cudaGetLastError();
  // number of key bits: keys of alive particles are < tiles * tr * tt; 0xFFFFFFFF must
  // sort after them, i.e. its low bits must exceed every alive key
  const int64_t ntr = (g.n_r + tr - 1) / tr, ntt = (g.n_th + tt - 1) / tt;
  const uint64_t maxkey = (uint64_t)ntr * ntt * tr * tt;  // exclusive bound
  int bits = 1;
  while (((uint64_t)1 << bits) - 1 < maxkey + 1 && bits < 32) ++bits;
  const int passes = (bits + 7) / 8;
  unsigned long long *alive = S.alive;
  cudaMemsetAsync(alive, 0, sizeof(unsigned long long), st);
  k_keys<T><<<grid_for(n_bound, TPB), TPB, 0, st>>>(in, g.n_r, tr, tt, S.keys[0], S.vals[0],
                                                     alive);
  COUNT_LAUNCH(1);
  const int nblocks = (int)((n_bound + BCHUNK - 1) / BCHUNK);
  const int64_t L = 256LL * nblocks;
  const int64_t nseg = (L + SCAN_SEG - 1) / SCAN_SEG;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_hist<<<nblocks, TPB, 0, st>>>(S.keys[cur], in.n, shift, nblocks, S.hist);
    COUNT_LAUNCH(1);
    k_scan_seg<<<(int)nseg, SCAN_SEG / 4, 0, st>>>(S.hist, L, S.bsum);
    COUNT_LAUNCH(1);
    k_scan_sums<<<1, SCAN_SUMS_TPB, 0, st>>>(S.bsum, nseg);
    COUNT_LAUNCH(1);
    k_scan_add<<<(int)((L + 255) / 256), 256, 0, st>>>(S.hist, L, S.bsum);
    COUNT_LAUNCH(1);
    k_scatter<<<nblocks, TPB, 0, st>>>(S.keys[cur], S.vals[cur], S.keys[1 - cur],
                                       S.vals[1 - cur], in.n, shift, nblocks, S.hist);
    COUNT_LAUNCH(1);
    cur = 1 - cur;
  }
  if (tile_start) {  // before k_set_n: the key count is the count before the sort
    const int n_tiles = (int)(ntr * ntt);
    k_tile_ranges<<<(n_tiles + 1 + 255) / 256, 256, 0, st>>>(S.keys[cur], in.n, n_tiles,
                                                             (uint32_t)(tr * tt), tile_start);
    COUNT_LAUNCH(1);
  }
  if (with_prev) k_gather<T, true><<<grid_for(n_bound, TPB), TPB, 0, st>>>(in, out, S.vals[cur], in.n);
  else k_gather<T, false><<<grid_for(n_bound, TPB), TPB, 0, st>>>(in, out, S.vals[cur], in.n);
  COUNT_LAUNCH(1);
  k_set_n<<<1, 1, 0, st>>>(n_dev, alive);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

template cudaError_t launch_sort<double>(const GridP &, int, int, SpeciesDevT<double>,
                                         SpeciesDevT<double>, int64_t, int64_t *,
                                         const SortScratch &, uint32_t *, cudaStream_t, bool);
template cudaError_t launch_sort<float>(const GridP &, int, int, SpeciesDevT<float>,
                                        SpeciesDevT<float>, int64_t, int64_t *,
                                        const SortScratch &, uint32_t *, cudaStream_t, bool);

// ---------------------------------------------------------------------------------
// grpic_sort_permutation_noalloc: the same stable cell sort, for callers that cannot
// provide scratch memory. Its scratch (key/index ping-pong buffers, digit histograms,
// scan sums, counters) is one file-scope device array below, shared by every call in
// the process on a given GPU.
// ---------------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int64_t NA_MAX = GRPIC_NOALLOC_SORT_MAX;
constexpr int64_t NA_BLOCKS = (NA_MAX + BCHUNK - 1) / BCHUNK;
constexpr int64_t NA_HIST = 256 * NA_BLOCKS;
constexpr int64_t NA_BSUM = (NA_HIST + SCAN_SEG - 1) / SCAN_SEG;
// byte offsets inside the scratch array (each a multiple of 256)
constexpr size_t NA_OFF_KEYS0 = 0;
constexpr size_t NA_OFF_KEYS1 = NA_OFF_KEYS0 + 4 * NA_MAX;
constexpr size_t NA_OFF_VALS0 = NA_OFF_KEYS1 + 4 * NA_MAX;
constexpr size_t NA_OFF_VALS1 = NA_OFF_VALS0 + 4 * NA_MAX;
constexpr size_t NA_OFF_HIST = NA_OFF_VALS1 + 4 * NA_MAX;
constexpr size_t NA_OFF_BSUM = NA_OFF_HIST + 4 * NA_HIST;
constexpr size_t NA_OFF_CNT = NA_OFF_BSUM + ((4 * NA_BSUM + 255) / 256) * 256;
constexpr size_t NA_BYTES = NA_OFF_CNT + 256;  // alive counter and element count

static __device__ __align__(256) unsigned char g_sort_scratch[NA_BYTES];

__global__ void k_store_count(int64_t *p, int64_t v) { *p = v; }

std::mutex g_na_mutex;
void *g_na_base[64] = {};

}  // namespace

extern "C" GRPIC_API grpic_status grpic_sort_permutation_noalloc(
    int n_r, int n_theta, int tile_r, int tile_theta, const int32_t *i1, const int32_t *i2,
    const uint8_t *tag, int64_t n, uint32_t *perm, int64_t *n_alive, void *stream) {
  if (n_r < 1 || n_theta < 1 || tile_r < 1 || tile_theta < 1 || n < 0) return GRPIC_EINVAL;
  if (n_r > 65536 || n_theta > 65536 || tile_r > 65536 || tile_theta > 65536)
    return GRPIC_EINVAL;
  // every key of a live particle (below the tile-padded cell count) must stay below the
  // dead key 0xFFFFFFFF and inside the int range the key arithmetic uses
  const int64_t ntr = (n_r + tile_r - 1) / tile_r, ntt = (n_theta + tile_theta - 1) / tile_theta;
  const uint64_t maxkey = (uint64_t)ntr * ntt * tile_r * tile_theta;
  if (maxkey > (uint64_t)INT32_MAX) return GRPIC_EINVAL;
  if (n > NA_MAX) return GRPIC_ECAPACITY;
  if (!n_alive || (n > 0 && (!i1 || !i2 || !tag || !perm))) return GRPIC_EINVAL;
  // an error left pending by earlier work on this thread is not this call's: leave it for
  // its owner to read and queue nothing
  if (cudaPeekAtLastError() != cudaSuccess) return GRPIC_ECUDA;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // set-up, once per device with that device current: the device address of the
  // scratch array (its host-side name is only a stand-in for it)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GRPIC_ECUDA;
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return GRPIC_ECUDA;
      g_na_base[dev] = p;
    }
    base = static_cast<unsigned char *>(g_na_base[dev]);
  }
  unsigned long long *alive = reinterpret_cast<unsigned long long *>(base + NA_OFF_CNT);
  int64_t *n_dev = reinterpret_cast<int64_t *>(base + NA_OFF_CNT + 8);
  if (n == 0) {
    k_store_count<<<1, 1, 0, st>>>(n_alive, 0);
    COUNT_LAUNCH(1);
    return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
  }
  uint32_t *keys[2] = {reinterpret_cast<uint32_t *>(base + NA_OFF_KEYS0),
                       reinterpret_cast<uint32_t *>(base + NA_OFF_KEYS1)};
  uint32_t *vals[2] = {reinterpret_cast<uint32_t *>(base + NA_OFF_VALS0),
                       reinterpret_cast<uint32_t *>(base + NA_OFF_VALS1)};
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + NA_OFF_HIST);
  uint32_t *bsum = reinterpret_cast<uint32_t *>(base + NA_OFF_BSUM);
  // the counter must start at zero: the array keeps the previous call's contents
  if (cudaMemsetAsync(alive, 0, sizeof(unsigned long long), st) != cudaSuccess) return GRPIC_ECUDA;
  k_store_count<<<1, 1, 0, st>>>(n_dev, n);
  SpeciesDevT<double> s{};
  s.i1 = const_cast<int32_t *>(i1);
  s.i2 = const_cast<int32_t *>(i2);
  s.tag = const_cast<uint8_t *>(tag);
  s.n = n_dev;
  int bits = 1;
  while (((uint64_t)1 << bits) - 1 < maxkey + 1 && bits < 32) ++bits;
  const int passes = (bits + 7) / 8;
  k_keys<double><<<grid_for(n, TPB), TPB, 0, st>>>(s, n_r, tile_r, tile_theta, keys[0], vals[0],
                                                   alive);
  const int nblocks = (int)((n + BCHUNK - 1) / BCHUNK);
  const int64_t L = 256LL * nblocks;
  const int64_t nseg = (L + SCAN_SEG - 1) / SCAN_SEG;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_hist<<<nblocks, TPB, 0, st>>>(keys[cur], n_dev, shift, nblocks, hist);
    k_scan_seg<<<(int)nseg, SCAN_SEG / 4, 0, st>>>(hist, L, bsum);
    k_scan_sums<<<1, SCAN_SUMS_TPB, 0, st>>>(bsum, nseg);
    k_scan_add<<<(int)((L + 255) / 256), 256, 0, st>>>(hist, L, bsum);
    k_scatter<<<nblocks, TPB, 0, st>>>(keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], n_dev,
                                       shift, nblocks, hist);
    cur = 1 - cur;
  }
  COUNT_LAUNCH(2 + 5 * passes);
  if (cudaMemcpyAsync(perm, vals[cur], (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GRPIC_ECUDA;
  k_set_n<<<1, 1, 0, st>>>(n_alive, alive);
  COUNT_LAUNCH(1);
  return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}
