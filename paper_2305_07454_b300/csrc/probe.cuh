// probe.cuh — binary64 issue-rate probe: the measured rate of the binary64 pipe (a part with
// about 2 binary64 operations per clock per SM), the roof of the FP64 form's journey kernels
// for the binary64 operations they keep (the coordinate differences, the cosines and the
// distance's final sum). Every thread runs kChains independent dependency chains of one operation
// kind, enough to keep the pipe's latency covered at a few warps per scheduler; the caller times
// the launch with CUDA events on its stream. Intrinsics with explicit rounding keep the compiler
// from fusing the mix's multiplies and adds into fma.
#pragma once
#include "common.cuh"

namespace cvetl {

constexpr int kProbeChains = 8;

enum ProbeKind { kProbeFma = 0, kProbeAdd = 1, kProbeMul = 2, kProbeMix = 3 };

// binary64 operations per chain per iteration of each kind: fma, add and mul one each; the mix
// is the journey kernel's per-point set (4 adds, 5 multiplies, 4 fma)
__host__ __device__ constexpr int probe_ops_per_iter(int kind) { return kind == kProbeMix ? 13 : 1; }

template <int Kind>
__global__ void __launch_bounds__(256) k_probe_fp64(long long iters, double b, double c, double* __restrict__ sink) {
  double a[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) {
      if constexpr (Kind == kProbeFma) {
        a[i] = fma(a[i], b, c);
      } else if constexpr (Kind == kProbeAdd) {
        a[i] = __dadd_rn(a[i], c);
      } else if constexpr (Kind == kProbeMul) {
        a[i] = __dmul_rn(a[i], b);
      } else {
        // 4 adds, 5 multiplies, 4 fma, as one chain per lane-chain
        double x = __dadd_rn(a[i], c);
        double y = __dmul_rn(x, b);
        double z = fma(y, b, c);
        x = __dadd_rn(z, -c);
        y = __dmul_rn(x, b);
        z = fma(y, b, -c);
        x = __dmul_rn(z, b);
        y = __dadd_rn(x, c);
        z = fma(y, b, c);
        x = __dmul_rn(z, b);
        y = __dadd_rn(x, -c);
        z = __dmul_rn(y, b);
        a[i] = fma(z, b, -c);
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace cvetl
