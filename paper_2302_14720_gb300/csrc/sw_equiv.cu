// sw_equiv.cu -- the paper's label-equivalence labelling (§2.3), kept as a
// comparator for the union-find path that the sweep uses.
//
// Labels start as the sites' own indices. Each iteration
//   scan:     every site takes the smallest label among itself and its
//             bonded neighbours (east, south, west, north) and, if that is
//             smaller than its own label l, proposes it for l's reference
//             (an atomic minimum on ref[l]);
//   analyse:  every reference is followed to the end of its chain, which
//             collapses the forest of references;
//   relabel:  every site takes the reference of its label.
// The loop ends when a scan proposes nothing; every site then holds the
// smallest index of its cluster, the same canonical label (C9) the tiled
// path writes. References only ever point to smaller labels, so every chain
// ends; the walk is capped all the same and the cap raises the error flag.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_internal.h"

namespace sw {
namespace {

constexpr int kChainCap = 1 << 24;

int grid_of(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

__global__ void le_init(int32_t* lab, int32_t* ref, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    lab[i] = (int32_t)i;
    ref[i] = (int32_t)i;
  }
}

__global__ void le_scan(const uint8_t* bonds, const int32_t* lab, int32_t* ref, int L, int* changed) {
  const int64_t n = (int64_t)L * L;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i - (int64_t)y * L);
    const int xe = x + 1 == L ? 0 : x + 1, xw = x == 0 ? L - 1 : x - 1;
    const int ys = y + 1 == L ? 0 : y + 1, yn = y == 0 ? L - 1 : y - 1;
    const int32_t l = lab[i];
    int32_t m = l;
    const uint8_t b = bonds[i];
    if (b & 1u) m = min(m, lab[(int64_t)y * L + xe]);
    if (b & 2u) m = min(m, lab[(int64_t)ys * L + x]);
    if (bonds[(int64_t)y * L + xw] & 1u) m = min(m, lab[(int64_t)y * L + xw]);
    if (bonds[(int64_t)yn * L + x] & 2u) m = min(m, lab[(int64_t)yn * L + x]);
    if (m < l) {
      atomicMin(ref + l, m);
      *changed = 1;
    }
  }
}

__global__ void le_analyse(int32_t* ref, int64_t n, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = ref[i];
    if (r == (int32_t)i) continue;
    for (int it = 0;; ++it) {
      const int32_t rr = ref[r];
      if (rr == r) break;
      if (it >= kChainCap) {
        atomicCAS(err, 0, 1);
        break;
      }
      r = rr;
    }
    ref[i] = r;
  }
}

__global__ void le_relabel(int32_t* lab, const int32_t* ref, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    lab[i] = ref[lab[i]];
}

}  // namespace

cudaError_t run_label_equivalence(const uint8_t* bonds, int L, int32_t* lab, int32_t* ref, int* d_changed, int* err,
                                  int max_iter, int* iterations, cudaStream_t st) {
  const int64_t n = (int64_t)L * L;
  const int g = grid_of(n, 256);
  le_init<<<g, 256, 0, st>>>(lab, ref, n);
  cudaError_t e = cudaGetLastError();
  int it = 0, changed = 1;
  while (e == cudaSuccess && changed && it < max_iter) {
    e = cudaMemsetAsync(d_changed, 0, sizeof(int), st);
    if (e == cudaSuccess) {
      le_scan<<<g, 256, 0, st>>>(bonds, lab, ref, L, d_changed);
      le_analyse<<<g, 256, 0, st>>>(ref, n, err);
      le_relabel<<<g, 256, 0, st>>>(lab, ref, n);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&changed, d_changed, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ++it;
  }
  *iterations = changed ? -it : it;  // negative: the cap was reached before convergence
  return e;
}

}  // namespace sw
