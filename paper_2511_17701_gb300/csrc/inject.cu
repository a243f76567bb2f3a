// inject.cu -- pair injection of the BZ monopole test (Sec. 4.5: plasma is injected wherever
// the local magnetization exceeds sigma_th).
//
// Per cell (i1 in [0, n_r), i2 in [0, n_th)): B at the cell centre from the em planes (B^1
// and B^2 averaged over the two faces, B^3 as stored), B_i B^i = h_ij B^i B^j with h at the
// centre, n = (sum of |w| of the live particles of both species in the cell) / sqrt(h) at
// the centre, sigma = sigma0 (B_i B^i / B0^2) / n. Where sigma > sigma_th one e- e+ pair is
// added at one point of the cell with weight dn sqrt(h_centre) / 2 each, dn the density that
// brings sigma down to sigma_th. Offsets and tetrad-frame momenta come from a caller's pool
// of random draws, 8 per pair, used in cell order from a cursor the library keeps; the k-th
// pair in cell order goes to slot n + k of both species, so the result does not depend on
// thread scheduling. When room runs out the first pairs in cell order are kept.
//
// Kernels: the density scatter (warp-reduced runs of equal cells, one FP64 atomic per run),
// the per-cell decision (FP64, with the cell-centre metric tabulated once per grid), an
// exclusive scan of the decisions (warp-shuffle block scans of 1024 cells, a scan of the
// block totals, a fix-up), the list of injecting cells, the writes of the new pairs (one
// thread per pair, so the FP64 metric and tetrad work runs in full warps) and the count
// update.
#include "grpic_internal.cuh"

namespace {

constexpr int SC_TPB = 256, SC_PER = 4, SC_BLOCK = SC_TPB * SC_PER;  // cells per scan block

// the metric at every cell centre, FP64, once per grid: [5][n_th][n_r] = h11, h22, h33, h13,
// sqrt(h) (the values the per-cell decision and the injected weights use)
constexpr int CT_H11 = 0, CT_H22 = 1, CT_H33 = 2, CT_H13 = 3, CT_SQH = 4, CT_ISQ = 5, CT_N = 6;
__global__ void k_inj_tables(GridP g, double *ct) {
  const int64_t nc = (int64_t)g.n_r * g.n_th;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n_r), j = (int)(c / g.n_r);
    MetricV m;
    metric_eval<false>(g, i + 0.5, j + 0.5, false, m, nullptr);
    ct[CT_H11 * nc + c] = m.h11;
    ct[CT_H22 * nc + c] = m.h22;
    ct[CT_H33 * nc + c] = m.h33;
    ct[CT_H13 * nc + c] = m.h13;
    ct[CT_SQH * nc + c] = m.sqrt_h;
    ct[CT_ISQ * nc + c] = 1.0 / m.sqrt_h;
  }
}

// summed |w| per cell. Particles are mostly sorted by cell, so consecutive lanes share a
// cell: each run of equal cells within the warp is summed by a suffix scan bounded by the
// next run head, and the head lane issues one atomic for the run.
template <typename T>
__global__ void k_inj_density(GridP g, SpeciesDevT<T> s, double *ncell) {
  const int64_t n = *s.n;
  const int lane = threadIdx.x & 31;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k - lane < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t cell = -1;
    double v = 0.0;
    if (k < n && s.tag[k] == 1) {
      const int i = s.i1[k], j = s.i2[k];
      if (i >= 0 && i < g.n_r && j >= 0 && j < g.n_th) {
        cell = (int64_t)j * g.n_r + i;
        v = fabs((double)s.w[k]);
      }
    }
    const int64_t prev = __shfl_up_sync(0xffffffffu, cell, 1);
    const bool head = lane == 0 || prev != cell;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const unsigned after = lane == 31 ? 0u : heads & ~((2u << lane) - 1u);
    const int end = after ? __ffs(after) - 1 : 32;
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_down_sync(0xffffffffu, v, o);
      if (lane + o < end) v += y;
    }
    if (head && cell >= 0) atomicAdd(ncell + cell, v);
  }
}

// B_i B^i at the centre of cell c = (i, j)
template <typename T>
__device__ __forceinline__ double cell_b2(const GridP &g, const T *const B[3], const double *ct,
                                          int64_t nc, int64_t c, int i, int j) {
  const int64_t k = sidx(g, i, j);
  const double b1 = 0.5 * ((double)B[0][k] + (double)B[0][k + 1]);
  const double b2 = 0.5 * ((double)B[1][k] + (double)B[1][k + g.NX]);
  const double b3 = (double)B[2][k];
  return ct[CT_H11 * nc + c] * b1 * b1 + ct[CT_H22 * nc + c] * b2 * b2 +
         ct[CT_H33 * nc + c] * b3 * b3 + 2.0 * ct[CT_H13 * nc + c] * b1 * b3;
}

// decision per cell: flag[c] = sigma > sigma_th; ncell[c] becomes dn (the density to add).
// The work is FP64 (GB300: 2 operations per clock per SM): no divisions, the constants
// st = sigma_th B0^2 and kd = sigma0 / (B0^2 sigma_th) come in from the host.
template <typename T>
__global__ void k_inj_decide(GridP g, FieldPtrsT<T> F, const double *ct, double *ncell,
                             uint32_t *flag, double sigma0, double st, double kd) {
  const int64_t nc = (int64_t)g.n_r * g.n_th;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n_r), j = (int)(c / g.n_r);
    const double b2 = cell_b2<T>(g, F.B, ct, nc, c, i, j);
    const double n = ncell[c] * ct[CT_ISQ * nc + c];
    const bool hot = sigma0 * b2 > st * n;  // sigma > sigma_th without dividing by n
    flag[c] = hot ? 1u : 0u;
    ncell[c] = hot ? kd * b2 - n : 0.0;
  }
}

// exclusive scan of the 256 threads' values; returns this thread's prefix, *total the sum
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t *warp_sums, uint32_t &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < SC_TPB / 32 ? warp_sums[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SC_TPB / 32) warp_sums[lane] = s;  // inclusive warp prefixes
  }
  __syncthreads();
  total = warp_sums[SC_TPB / 32 - 1];
  const uint32_t before = w ? warp_sums[w - 1] : 0u;
  __syncthreads();
  return before + x - v;
}

// per block of SC_BLOCK values: exclusive scan in place, block total to bsum
__global__ void __launch_bounds__(SC_TPB) k_scan_block(uint32_t *a, int64_t L, uint32_t *bsum) {
  __shared__ uint32_t ws[SC_TPB / 32];
  const int64_t base = (int64_t)blockIdx.x * SC_BLOCK + (int64_t)threadIdx.x * SC_PER;
  uint32_t v[SC_PER], sum = 0;
  for (int q = 0; q < SC_PER; ++q) {
    v[q] = base + q < L ? a[base + q] : 0u;
    sum += v[q];
  }
  uint32_t total;
  uint32_t run = block_scan(sum, ws, total);
  for (int q = 0; q < SC_PER; ++q) {
    if (base + q < L) a[base + q] = run;
    run += v[q];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// one block: exclusive scan of the block totals in place (chunks of SC_BLOCK with a carry),
// the grand total to *total
__global__ void __launch_bounds__(SC_TPB) k_scan_totals(uint32_t *bsum, int64_t nb,
                                                        uint32_t *total) {
  __shared__ uint32_t ws[SC_TPB / 32];
  uint32_t carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += SC_BLOCK) {
    const int64_t base = c0 + (int64_t)threadIdx.x * SC_PER;
    uint32_t v[SC_PER], sum = 0;
    for (int q = 0; q < SC_PER; ++q) {
      v[q] = base + q < nb ? bsum[base + q] : 0u;
      sum += v[q];
    }
    uint32_t chunk;
    uint32_t run = carry + block_scan(sum, ws, chunk);
    for (int q = 0; q < SC_PER; ++q) {
      if (base + q < nb) bsum[base + q] = run;
      run += v[q];
    }
    carry += chunk;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_fix(uint32_t *a, int64_t L, const uint32_t *bsum) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < L;
       t += (int64_t)gridDim.x * blockDim.x)
    a[t] += bsum[t / SC_BLOCK];
}

// the cells that inject, in cell order: cell c injects iff its exclusive offset steps up
__global__ void k_inj_list(int64_t nc, const uint32_t *off, const uint32_t *total,
                           uint32_t *list) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = off[c], next = c + 1 < nc ? off[c + 1] : *total;
    if (next != k) list[k] = (uint32_t)c;
  }
}

// the new pairs, one thread per pair (full warps for the FP64 metric and tetrads): pair k
// of cell list[k] goes to slot n + k of both species if k < room
template <typename T>
__global__ void k_inj_write(GridP g, SpeciesDevT<T> se, SpeciesDevT<T> sp, int64_t cap_e,
                            int64_t cap_p, const uint32_t *list, const uint32_t *total,
                            const double *dn, const double *ct, const double *pool,
                            int64_t pool_n, const int64_t *cursor) {
  const int64_t nc = (int64_t)g.n_r * g.n_th;
  const int64_t ne = *se.n, np = *sp.n;
  const int64_t room = cap_e - ne < cap_p - np ? cap_e - ne : cap_p - np;
  const int64_t t = (int64_t)*total, npairs = t < room ? t : room;
  const int64_t cur = *cursor;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < npairs;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = list[k];
    const int i = (int)(c % g.n_r), j = (int)(c / g.n_r);
    const double *r = pool + 8 * ((cur + k) % pool_n);
    const double w = 0.5 * dn[c] * ct[CT_SQH * nc + c];
    MetricV m;
    metric_eval<false>(g, i + r[0], j + r[1], true, m, nullptr);
    for (int q = 0; q < 2; ++q) {
      const SpeciesDevT<T> &s = q ? sp : se;
      const int64_t p = (q ? np : ne) + k;
      const double uh[3] = {r[2 + 3 * q], r[3 + 3 * q], r[4 + 3 * q]};
      double u[3];
      t_hat_to_cov(m, uh, u);
      s.i1[p] = i; s.i2[p] = j;
      s.dx1[p] = (T)r[0]; s.dx2[p] = (T)r[1];
      s.u1[p] = (T)u[0]; s.u2[p] = (T)u[1]; s.u3[p] = (T)u[2];
      s.w[p] = (T)w;
      s.phi[p] = (T)0;
      s.tag[p] = 1;
      s.i1p[p] = i; s.i2p[p] = j; s.dx1p[p] = s.dx1[p]; s.dx2p[p] = s.dx2[p];
    }
  }
}

template <typename T>
__global__ void k_inj_finish(SpeciesDevT<T> se, SpeciesDevT<T> sp, int64_t cap_e, int64_t cap_p,
                             const uint32_t *total, int64_t *cursor, int64_t pool_n,
                             unsigned long long *diag) {
  const int64_t ne = *se.n, np = *sp.n;
  const int64_t room = cap_e - ne < cap_p - np ? cap_e - ne : cap_p - np;
  const int64_t t = (int64_t)*total, added = t < room ? t : room;
  *const_cast<int64_t *>(se.n) = ne + added;  // the count lives in the arena
  *const_cast<int64_t *>(sp.n) = np + added;
  *cursor = (*cursor + added) % pool_n;
  diag[DG_INJECTED] += (unsigned long long)added;
  diag[DG_INJECT_DROPPED] += (unsigned long long)(t - added);
}

__global__ void k_inj_cursor(int64_t *cursor, int64_t v) { *cursor = v; }

int blocks_of(int64_t n, int tpb) {
  int64_t b = (n + tpb - 1) / tpb;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

size_t inject_scratch_bytes(const GridP &g) {
  const int64_t nc = (int64_t)g.n_r * g.n_th;
  const int64_t nb = (nc + SC_BLOCK - 1) / SC_BLOCK;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  return up(nc * 8) + up(nc * 4) + up((nb + 1) * 4) + up(64) + up(CT_N * nc * 8) + up(nc * 4);
}

// the cell-centre metric table at the end of the scratch (grpic_init_metric)
cudaError_t launch_inject_tables(const GridP &g, unsigned char *scratch, cudaStream_t st) {
  const int64_t nc = (int64_t)g.n_r * g.n_th;
  const int64_t nb = (nc + SC_BLOCK - 1) / SC_BLOCK;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  double *ct = reinterpret_cast<double *>(scratch + up(nc * 8) + up(nc * 4) + up((nb + 1) * 4) +
                                          up(64));
  k_inj_tables<<<blocks_of(nc, 256), 256, 0, st>>>(g, ct);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inject(const GridP &g, const FieldPtrsT<T> &F, SpeciesDevT<T> se,
                          SpeciesDevT<T> sp, int64_t n_bound_e, int64_t n_bound_p,
                          int64_t cap_e, int64_t cap_p, double sigma0, double sigma_th,
                          double B0, const double *pool, int64_t pool_n, int64_t pool_offset,
                          unsigned char *scratch, unsigned long long *diag, cudaStream_t st) {
  const int64_t nc = (int64_t)g.n_r * g.n_th;
  const int64_t nb = (nc + SC_BLOCK - 1) / SC_BLOCK;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  double *ncell = reinterpret_cast<double *>(scratch);
  uint32_t *flag = reinterpret_cast<uint32_t *>(scratch + up(nc * 8));
  uint32_t *bsum = reinterpret_cast<uint32_t *>(scratch + up(nc * 8) + up(nc * 4));
  unsigned char *tail = scratch + up(nc * 8) + up(nc * 4) + up((nb + 1) * 4);
  int64_t *cursor = reinterpret_cast<int64_t *>(tail);
  uint32_t *total = reinterpret_cast<uint32_t *>(tail + 8);
  const double *ct = reinterpret_cast<const double *>(tail + up(64));
  uint32_t *list = reinterpret_cast<uint32_t *>(tail + up(64) + up(CT_N * nc * 8));
  if (pool_offset >= 0) {
    k_inj_cursor<<<1, 1, 0, st>>>(cursor, pool_offset % pool_n);
    COUNT_LAUNCH(1);
  }
  cudaError_t e = cudaMemsetAsync(ncell, 0, nc * 8, st);
  if (e != cudaSuccess) return e;
  if (n_bound_e > 0) {
    k_inj_density<T><<<blocks_of(n_bound_e, 256), 256, 0, st>>>(g, se, ncell);
    COUNT_LAUNCH(1);
  }
  if (n_bound_p > 0) {
    k_inj_density<T><<<blocks_of(n_bound_p, 256), 256, 0, st>>>(g, sp, ncell);
    COUNT_LAUNCH(1);
  }
  k_inj_decide<T><<<blocks_of(nc, 256), 256, 0, st>>>(g, F, ct, ncell, flag, sigma0,
                                                      sigma_th * B0 * B0,
                                                      sigma0 / (B0 * B0 * sigma_th));
  k_scan_block<<<(int)nb, SC_TPB, 0, st>>>(flag, nc, bsum);
  k_scan_totals<<<1, SC_TPB, 0, st>>>(bsum, nb, total);
  k_scan_fix<<<blocks_of(nc, 256), 256, 0, st>>>(flag, nc, bsum);
  k_inj_list<<<blocks_of(nc, 256), 256, 0, st>>>(nc, flag, total, list);
  // the pair count is on the device: enough blocks for one pair per cell, idle past it
  k_inj_write<T><<<blocks_of(nc, 128), 128, 0, st>>>(g, se, sp, cap_e, cap_p, list, total, ncell,
                                                     ct, pool, pool_n, cursor);
  k_inj_finish<T><<<1, 1, 0, st>>>(se, sp, cap_e, cap_p, total, cursor, pool_n, diag);
  COUNT_LAUNCH(7);
  return cudaGetLastError();
}

#define INSTANTIATE_INJECT(T)                                                                  \
  template cudaError_t launch_inject<T>(const GridP &, const FieldPtrsT<T> &, SpeciesDevT<T>,   \
                                        SpeciesDevT<T>, int64_t, int64_t, int64_t, int64_t,     \
                                        double, double, double, const double *, int64_t,        \
                                        int64_t, unsigned char *, unsigned long long *,         \
                                        cudaStream_t);
INSTANTIATE_INJECT(double)
INSTANTIATE_INJECT(float)
