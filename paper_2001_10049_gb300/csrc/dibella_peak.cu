// Integer-throughput microbenchmark: the measured ceiling that the extension
// kernels' cell rates are compared with.
//
// Every thread runs kChains independent dependency chains of one instruction
// class for `iters` iterations, on a grid that fills every SM to its occupancy
// limit, so the measured rate is the issue/pipe throughput of that class and
// not a latency.  The operands come from registers set from the thread index
// at run time and the results are folded into one store, so the compiler can
// neither evaluate nor drop the chains.  Classes:
//   0  IADD      x = (x + y) + z                   (2 instructions, 2 ops)
//   1  IMNMX     x = min(max(x, y), z)             (2 instructions, 2 ops)
//   2  VIADDMNMX x = max(x + y, z), int16 pairs    (2 ops x 2 halves = 4)
//   3  VIMNMX3   x = min(x, y, z), int16 pairs     (2 x 2 = 4)
//   4  cell      one int32 DP cell with the 8 ops of the cell convention:
//                diagonal compare + select + add, gap max + add, final max,
//                prune compare + select (8 ops)
// The entry point reports lane-ops per second (class 4: cells per second x 8).
// The paper has no counterpart: this is measurement infrastructure.

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dibella.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// Never written in practice; it only gives the kernels a valid address.
__device__ unsigned g_peak_sink;

template <int C>
__global__ void __launch_bounds__(kThreads) int_peak_kernel(long long iters, unsigned seed, unsigned* sink) {
  const unsigned t = threadIdx.x + blockIdx.x * blockDim.x;
  unsigned x[kChains], y[kChains], z[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = (t * 2654435761u) ^ (seed + 97u * c);
    y[c] = (t + 7u * c) ^ (seed >> 3);
    z[c] = (t * 40503u + c) ^ seed;
  }
  const int M = (int)(seed & 1u) + 1, S = -(int)((seed >> 1) & 1u) - 1, G = -(int)((seed >> 2) & 1u) - 1;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (C == 0) {
        // two dependent adds per chain; inline PTX keeps the compiler from
        // summing the linear recurrence in closed form
        asm volatile("add.s32 %0, %0, %1;" : "+r"(x[c]) : "r"(y[c]));
        asm volatile("add.s32 %0, %0, %1;" : "+r"(x[c]) : "r"(z[c]));
      } else if (C == 1) {
        int v = (int)x[c];
        asm volatile("max.s32 %0, %0, %1;" : "+r"(v) : "r"((int)y[c]));
        asm volatile("min.s32 %0, %0, %1;" : "+r"(v) : "r"((int)z[c]));
        x[c] = (unsigned)v;
      } else if (C == 2) {
        x[c] = __viaddmax_s16x2(x[c], y[c], z[c]);
        y[c] = __viaddmax_s16x2(y[c], z[c], x[c]);
      } else if (C == 3) {
        x[c] = __vimin3_s16x2(x[c], y[c], z[c]);
        y[c] = __vimax3_s16x2(y[c], z[c], x[c]);
      } else {
        // x = H(d-1) neighbour chain, y = diagonal, z = the other neighbour and
        // the base bits; thr from the seed.  The result feeds the next cell.
        const int u = (int)x[c], dg = (int)y[c], lf = (int)z[c];
        const int sub = ((z[c] ^ (unsigned)i) & 3u) == 0u ? M : S;
        int h = max(max(u, lf) + G, dg + sub);
        h = h >= (int)seed - 64 ? h : -(1 << 29);
        y[c] = x[c];
        x[c] = (unsigned)h;
      }
    }
  }
  unsigned acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= x[c] ^ y[c];
  if (acc == 0x9E3779B9u) sink[0] = acc;  // practically never taken; keeps the chains live
}

template <int C>
cudaError_t launch(int grid, long long iters, unsigned seed, unsigned* sink, cudaStream_t st) {
  int_peak_kernel<C><<<grid, kThreads, 0, st>>>(iters, seed, sink);
  return cudaGetLastError();
}

// Lane-operations per thread per iteration of each class (see the table above).
constexpr double kOpsPerIter[5] = {kChains * 2.0, kChains * 2.0, kChains * 2.0 * 4.0, kChains * 2.0 * 4.0,
                                   kChains * 8.0};

}  // namespace

extern "C" {

int dibella_int_peak(int32_t op_class, int64_t iters, double* ops_per_s_out, double* ms_out, void* stream) {
  if (op_class < 0 || op_class > 4 || iters < 1 || iters > (1ll << 30) || !ops_per_s_out) return DIBELLA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return DIBELLA_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DIBELLA_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DIBELLA_ECUDA;
  const void* fns[5] = {(const void*)int_peak_kernel<0>, (const void*)int_peak_kernel<1>,
                        (const void*)int_peak_kernel<2>, (const void*)int_peak_kernel<3>,
                        (const void*)int_peak_kernel<4>};
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[op_class], kThreads, 0) != cudaSuccess)
    return DIBELLA_ECUDA;
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  unsigned* sink = nullptr;
  if (cudaGetSymbolAddress((void**)&sink, g_peak_sink) != cudaSuccess) return DIBELLA_ECUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DIBELLA_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DIBELLA_ECUDA;
  }
  const unsigned seed = 0x5bd1e995u;
  cudaError_t e = cudaSuccess;
  float ms = 0;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first launch warms up
    cudaEventRecord(e0, st);
    switch (op_class) {
      case 0: e = launch<0>(grid, iters, seed, sink, st); break;
      case 1: e = launch<1>(grid, iters, seed, sink, st); break;
      case 2: e = launch<2>(grid, iters, seed, sink, st); break;
      case 3: e = launch<3>(grid, iters, seed, sink, st); break;
      default: e = launch<4>(grid, iters, seed, sink, st); break;
    }
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0) return DIBELLA_ECUDA;
  *ops_per_s_out = (double)grid * kThreads * (double)iters * kOpsPerIter[op_class] / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return DIBELLA_OK;
}

}  // extern "C"
