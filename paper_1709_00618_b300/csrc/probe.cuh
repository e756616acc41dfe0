// Issue-rate probes of the FMA pipes, used as the measured denominators of
// the Kalman kernels' ALU rooflines: every thread runs 8 independent chains
// of fused multiply-adds (enough in flight to cover the pipe latency).
#pragma once
#include "common.cuh"

namespace tpc {

constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
  T v[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; k++) v[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) v[k] = fma(v[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; k++) s += v[k];
  if (s == (T)-1.2345) out[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace tpc
