// Seeded synthetic workload generator: R-MAT edge lists, edge weights,
// personalized-PageRank seed sets and target sets.
//
// This module produces INPUTS only. It holds none of the graph method's
// arithmetic, and both the FP64 oracle tests and the CUDA path consume what it
// writes. The host and device versions below implement one definition and are
// bit-identical (tests check this).
//
// Random stream: the SplitMix64 output function (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a
// counter. Draw number k of stream s is
//     u(s, k) = mix64(mix64(s + GAMMA) + (k + 1) * GAMMA),  GAMMA = 0x9E3779B97F4A7C15.
// R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): edge e of a graph with
// seed S and 2^scale vertices takes, at bit level l = 0 .. scale-1 (most
// significant first), the draw u(S, 64*e + l) and picks the quadrant
// (src bit, dst bit) = (0,0) if u < TA, (0,1) if u < TAB, (1,0) if u < TABC,
// else (1,1), where TA/TAB/TABC are the cumulative probabilities a, a+b, a+b+c
// scaled to 2^64. No noise and no vertex permutation; duplicates and
// self-loops are kept.
// Edge weight e: w = 0.5 + (u(S, 64*e + 63) >> 41) * 2^-23, exactly
// representable in FP32, uniform on [0.5, 1.5).
#include <cstdint>
#include <cuda_runtime.h>

#define RMAT_GAMMA 0x9E3779B97F4A7C15ull

__host__ __device__ static inline uint64_t rmat_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ static inline uint64_t rmat_draw(uint64_t key, uint64_t k) {
  return rmat_mix64(key + (k + 1) * RMAT_GAMMA);
}

__host__ __device__ static inline void rmat_edge(uint64_t key, uint64_t e, int scale, uint64_t ta,
                                                 uint64_t tab, uint64_t tabc, uint32_t* s,
                                                 uint32_t* d) {
  uint32_t src = 0, dst = 0;
  for (int l = 0; l < scale; ++l) {
    uint64_t u = rmat_draw(key, 64ull * e + (uint64_t)l);
    uint32_t sb = (u >= tab) ? 1u : 0u;
    uint32_t db = (u >= ta && u < tab) || (u >= tabc) ? 1u : 0u;
    src = (src << 1) | sb;
    dst = (dst << 1) | db;
  }
  *s = src;
  *d = dst;
}

__host__ __device__ static inline float rmat_weight(uint64_t key, uint64_t e) {
  uint64_t u = rmat_draw(key, 64ull * e + 63ull);
  return (float)(0.5 + (double)(u >> 41) * (1.0 / 8388608.0));
}

__global__ void rmat_kernel(uint64_t key, uint64_t e0, uint64_t count, int scale, uint64_t ta,
                            uint64_t tab, uint64_t tabc, uint32_t* src, uint32_t* dst, float* w) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
    uint64_t e = e0 + t;
    uint32_t s, d;
    rmat_edge(key, e, scale, ta, tab, tabc, &s, &d);
    src[t] = s;
    dst[t] = d;
    if (w) w[t] = rmat_weight(key, e);
  }
}

extern "C" {

// Fill src[0..count), dst[0..count) (and w if non-null) with edges e0 .. e0+count-1.
// Host memory; OpenMP-parallel. Returns 0.
int rmat_generate_host(uint64_t seed, int scale, uint64_t e0, uint64_t count, uint64_t ta,
                       uint64_t tab, uint64_t tabc, uint32_t* src, uint32_t* dst, float* w) {
  uint64_t key = rmat_mix64(seed + RMAT_GAMMA);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < (int64_t)count; ++t) {
    uint32_t s, d;
    rmat_edge(key, e0 + (uint64_t)t, scale, ta, tab, tabc, &s, &d);
    src[t] = s;
    dst[t] = d;
    if (w) w[t] = rmat_weight(key, e0 + (uint64_t)t);
  }
  return 0;
}

// Same stream into device memory on `stream` (a cudaStream_t, may be null).
// Returns the cudaError_t of the launch.
int rmat_generate_device(uint64_t seed, int scale, uint64_t e0, uint64_t count, uint64_t ta,
                         uint64_t tab, uint64_t tabc, uint32_t* src, uint32_t* dst, float* w,
                         void* stream) {
  if (count == 0) return 0;
  uint64_t key = rmat_mix64(seed + RMAT_GAMMA);
  uint64_t blocks = (count + 255) / 256;
  if (blocks > 148ull * 64) blocks = 148ull * 64;
  rmat_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(key, e0, count, scale, ta, tab,
                                                                  tabc, src, dst, w);
  return (int)cudaGetLastError();
}

// Raw draws u(seed, k0 .. k0+count-1) (host), used for seed/target sets.
int rmat_draws_host(uint64_t seed, uint64_t k0, uint64_t count, uint64_t* out) {
  uint64_t key = rmat_mix64(seed + RMAT_GAMMA);
  for (uint64_t t = 0; t < count; ++t) out[t] = rmat_draw(key, k0 + t);
  return 0;
}

}  // extern "C"
