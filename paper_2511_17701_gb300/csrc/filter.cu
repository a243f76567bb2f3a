// filter.cu -- the current filter applied after the deposit (Sec. 3.2: deposition is followed
// by n_f filter passes; Sec. 3.3.3: the horizon layer i1 <= n_f is sized by them).
//
// One pass replaces each value by the binomial (1 2 1) x (1 2 1) / 16 stencil on the grid
// extended across each axis by the mirror image of the particles: node-row quantities (J^1,
// J^3, rho) are even and half-row ones (J^2) odd across an axis, and an axis node, which
// holds the charge of a half cell, holds twice that in the extended grid. Values beyond the
// stored x1 range read as zero; rows outside a component's range are zero on output. The
// filter commutes with the differences of the discrete continuity equation, so filtered
// currents conserve the filtered charge.
//
// GB300 layout: one CTA per 64 x 32 output tile and component. The tile and a halo of P
// cells (P <= 8 passes per launch) are loaded once, already extended across the axes; the P
// passes run in shared memory (the valid region shrinking by one cell per pass) and the
// centre is written once: 2 plane sweeps of HBM traffic for up to 8 passes. The FP64 form is
// bound by GB300's FP64 pipe, so each pass is the stencil's two factors, (1 2 1) along x1
// into a second buffer and (1 2 1) along x2 back, two operations per cell and factor, with
// the 1/16 per pass applied once at the end (powers of two: exact). The sums run in the
// order of the plain definition, so every result has the same bits.
#include "grpic_internal.cuh"

namespace {

constexpr int FT_X = 64, FT_Y = 32, F_MAXP = 8, F_TPB = 512;

template <typename T>
struct FilterPlanes {
  const T *in[3];
  T *out[3];
  int half[3];    // 1: half rows (x2 = j + 1/2)
  T parity[3];    // +1 even, -1 odd across the axes
};

// the stored row holding extended row j of a component, with the sign and axis factor f;
// -1 for a row more than 64 reflections away (never one a written row depends on)
__device__ __forceinline__ int reflect_row(int j, int N, int half, float par, float &f) {
  f = 1.0f;
  for (int k = 0; k < 64; ++k) {
    if (!half) {
      if (j < 0) { j = -j; f *= par; continue; }
      if (j > N) { j = 2 * N - j; f *= par; continue; }
    } else {
      if (j < 0) { j = -j - 1; f *= par; continue; }
      if (j > N - 1) { j = 2 * N - j - 1; f *= par; continue; }
    }
    if (!half && (j == 0 || j == N)) f *= 2.0f;
    return j;
  }
  return -1;
}

template <typename T>
size_t filter_smem(int P) {
  return (size_t)2 * (FT_X + 2 * P) * (FT_Y + 2 * P) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(F_TPB) k_filter(GridP g, FilterPlanes<T> fp, int P) {
  extern __shared__ unsigned char f_smem[];
  const int W = FT_X + 2 * P, H = FT_Y + 2 * P;
  T *A = reinterpret_cast<T *>(f_smem), *Bt = A + W * H;  // values, x1 sums
  const int c = blockIdx.z;
  const T *in = fp.in[c];
  T *out = fp.out[c];
  const int half = fp.half[c];
  const float par = (float)fp.parity[c];
  const int N = g.n_th;
  const int i0 = -G_ + (int)blockIdx.x * FT_X, j0 = -G_ + (int)blockIdx.y * FT_Y;  // stored
  const int ilo = -G_, ihi = g.n_r + G_;
  // load the extended values of the tile and its halo; cells beyond the x1 range are zero
  for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
    const int ly = e / W, lx = e - ly * W;
    const int i = i0 - P + lx, j = j0 - P + ly;
    T v = (T)0;
    if (i >= ilo && i <= ihi) {
      float f;
      const int jr = reflect_row(j, N, half, par, f);
      if (jr >= 0) v = (T)f * in[sidx(g, i, jr)];
    }
    A[e] = v;
  }
  __syncthreads();
  for (int p = 1; p <= P; ++p) {
    // along x1, rows p-1 .. H-p, columns p .. W-p-1; zero beyond the stored x1 range
    const int w = W - 2 * p, h1 = H - 2 * p + 2;
    for (int e = threadIdx.x; e < w * h1; e += blockDim.x) {
      const int ly = p - 1 + e / w, lx = p + e % w;
      const int i = i0 - P + lx;
      const T *a = A + ly * W + lx;
      Bt[ly * W + lx] = (i >= ilo && i <= ihi) ? (a[-1] + (T)2 * a[0]) + a[1] : (T)0;
    }
    __syncthreads();
    // along x2, rows p .. H-p-1
    const int h = H - 2 * p;
    for (int e = threadIdx.x; e < w * h; e += blockDim.x) {
      const int ly = p + e / w, lx = p + e % w;
      const T *b = Bt + ly * W + lx;
      A[ly * W + lx] = (b[-W] + (T)2 * b[0]) + b[W];
    }
    __syncthreads();
  }
  // the centre tile back to stored values: 16^-P, and the axis node rows hold half cells
  T scale = (T)1;
  for (int p = 0; p < P; ++p) scale *= (T)0.0625;
  const int jmax = half ? N - 1 : N;
  for (int e = threadIdx.x; e < FT_X * FT_Y; e += blockDim.x) {
    const int ty = e / FT_X, tx = e - ty * FT_X;
    const int i = i0 + tx, j = j0 + ty;
    if (i > ihi || j > N + G_) continue;
    T v = (T)0;
    if (j >= 0 && j <= jmax) {
      v = A[(P + ty) * W + P + tx] * scale;
      if (!half && (j == 0 || j == N)) v *= (T)0.5;
    }
    out[sidx(g, i, j)] = v;
  }
}

template <typename T>
cudaError_t filter_chunk(const GridP &g, const FilterPlanes<T> &fp, int n_comp, int P,
                         cudaStream_t st) {
  static bool attr = false;  // per instantiation: opt in to the largest tile's shared memory
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_filter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)filter_smem<T>(F_MAXP));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((g.NX + FT_X - 1) / FT_X, (g.NY + FT_Y - 1) / FT_Y, n_comp);
  k_filter<T><<<grid, F_TPB, filter_smem<T>(P), st>>>(g, fp, P);
  COUNT_LAUNCH(1);
  return cudaGetLastError();
}

}  // namespace

// n passes on n_comp (<= 3) planes: a[c] in; s[c] are scratch planes of the same size.
// Passes run in chunks of at most 8 per launch, alternating between a and s. When the last
// chunk ends in s, *in_s (if given) is set and the caller takes the result from s;
// otherwise (in_s null) it is copied back into a.
template <typename T>
cudaError_t launch_filter(const GridP &g, T *const a[3], T *const s[3], const int half[3],
                          const double parity[3], int n_comp, int n, cudaStream_t st,
                          bool *in_s) {
  if (in_s) *in_s = false;
  if (n <= 0 || n_comp <= 0) return cudaSuccess;
  FilterPlanes<T> fp{};
  bool in_a = true;
  for (int done = 0; done < n;) {
    const int P = n - done < F_MAXP ? n - done : F_MAXP;
    for (int c = 0; c < n_comp; ++c) {
      fp.in[c] = in_a ? a[c] : s[c];
      fp.out[c] = in_a ? s[c] : a[c];
      fp.half[c] = half[c];
      fp.parity[c] = (T)parity[c];
    }
    cudaError_t e = filter_chunk<T>(g, fp, n_comp, P, st);
    if (e != cudaSuccess) return e;
    in_a = !in_a;
    done += P;
  }
  if (!in_a && in_s) {
    *in_s = true;
    return cudaSuccess;
  }
  if (!in_a) {
    const size_t bytes = (size_t)g.NX * g.NY * sizeof(T);
    for (int c = 0; c < n_comp; ++c) {
      cudaError_t e = cudaMemcpyAsync(a[c], s[c], bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// the n_f passes on the currents J^1 (node rows, even), J^2 (half rows, odd), J^3 (node
// rows, even), with the auxiliary E planes (scratch between uses) as the other buffer; when
// the result lands there the two sets of planes trade places (no copy)
template <typename T>
cudaError_t launch_filter_currents(const GridP &g, FieldPtrsT<T> &F, cudaStream_t st) {
  const int half[3] = {0, 1, 0};
  const double par[3] = {1.0, -1.0, 1.0};
  bool in_s = false;
  cudaError_t e = launch_filter<T>(g, F.J, F.E, half, par, 3, g.n_f, st, &in_s);
  if (e == cudaSuccess && in_s)
    for (int c = 0; c < 3; ++c) {
      T *t = F.J[c];
      F.J[c] = F.E[c];
      F.E[c] = t;
    }
  return e;
}

#define INSTANTIATE_FILTER(T)                                                                  \
  template cudaError_t launch_filter<T>(const GridP &, T *const[3], T *const[3], const int[3],  \
                                        const double[3], int, int, cudaStream_t, bool *);       \
  template cudaError_t launch_filter_currents<T>(const GridP &, FieldPtrsT<T> &, cudaStream_t);
INSTANTIATE_FILTER(double)
INSTANTIATE_FILTER(float)
