// probe.cu -- throughput probe of the arithmetic pipes that bound the pusher kernels (no
// counterpart in the paper; it supplies the measured denominators of their rooflines).
//
// The FP64 pusher is bound by the FP64 pipe, the mixed one by instruction issue. Each thread
// of the probe runs CHAINS independent chains of one arithmetic operation (fused
// multiply-add a = a b + c, multiply a = a b or add a = a + c), UNROLL of them per loop trip,
// so the loop's bookkeeping is a few instructions in CHAINS x UNROLL and the chains hide the
// pipe's latency. In FP64 the launch runs at the FP64 pipe's rate for that operation; in FP32
// every operation is one lane of a warp instruction that the FP32 pipe takes at one per
// clock and SM sub-partition, which is also the issue rate, so the FP32 figure is the SM's
// warp instruction peak (times 32 lanes).
#include "grpic_internal.cuh"

namespace {

constexpr int PROBE_TPB = 256;
constexpr int CHAINS = 8;
constexpr int UNROLL = 32;

template <typename R, int OP>
__global__ void __launch_bounds__(PROBE_TPB) k_probe(int64_t iters, R b, R c, double *sink) {
  R a[CHAINS];
#pragma unroll
  for (int q = 0; q < CHAINS; ++q) a[q] = (R)(threadIdx.x + q + 1) * (R)1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int q = 0; q < CHAINS; ++q) {
        if (OP == 0) a[q] = fma(a[q], b, c);
        else if (OP == 1) a[q] = a[q] * b;
        else a[q] = a[q] + c;
      }
  }
  R t = (R)0;
#pragma unroll
  for (int q = 0; q < CHAINS; ++q) t += a[q];
  // every chain stays positive (b = 1 - 2^-20 > 0, c > 0, positive starts), so this store
  // never happens; the compiler cannot know that and keeps every operation
  if (t == (R)-1) *sink = (double)t;
}

template <typename R>
void launch_probe(int op, int blocks, cudaStream_t st, int64_t iters, R b, R c, double *sink) {
  if (op == 0) k_probe<R, 0><<<blocks, PROBE_TPB, 0, st>>>(iters, b, c, sink);
  else if (op == 1) k_probe<R, 1><<<blocks, PROBE_TPB, 0, st>>>(iters, b, c, sink);
  else k_probe<R, 2><<<blocks, PROBE_TPB, 0, st>>>(iters, b, c, sink);
}

}  // namespace

extern "C" GRPIC_API grpic_status grpic_probe_alu(int precision, int op, int64_t iters,
                                                  int blocks_per_sm, double *sink, void *stream,
                                                  int64_t *ops) {
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || !sink || !ops) return GRPIC_EINVAL;
  if (op < 0 || op > 2) return GRPIC_EINVAL;
  if (precision != GRPIC_FP64 && precision != GRPIC_MIXED) return GRPIC_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return GRPIC_ECUDA;  // not this call's error
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return GRPIC_ECUDA;
  const int blocks = sms * blocks_per_sm;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == GRPIC_FP64) launch_probe<double>(op, blocks, st, iters, 1.0 - 0x1p-20, 0x1p-20, sink);
  else launch_probe<float>(op, blocks, st, iters, 1.0f - 0x1p-20f, 0x1p-20f, sink);
  COUNT_LAUNCH(1);
  *ops = (int64_t)blocks * PROBE_TPB * CHAINS * UNROLL * iters;
  return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}
