// Helpers shared by the geometry-term translation units (grid edges,
// regularizers, Marching Tetrahedra): the workspace status block, a
// device-wide exclusive scan of int counts, and grid sizing.  Everything has
// internal linkage, so each translation unit holds its own copy.
#pragma once

#include <algorithm>

#include "geometry.cuh"

namespace tts {

// launch counter shared with the other entry points (api.cu)
void count_launches(long long n);

namespace {

constexpr int RT = 256;          // threads per block
constexpr int SCAN_T = 1024;     // scan block size
constexpr int SCAN_CHUNK = 4096; // elements per scan block

// Status block at the start of every geometry-term workspace.
struct GeoStatus {
  unsigned int status;
  unsigned int pad[3];
  long long total;               // last scan total
  long long counts[2];           // Marching Tetrahedra vertex / triangle totals
  double acc[2];                 // L_eik, L_nc accumulators
};

__device__ __forceinline__ bool valid4(int4 t, long long N) {
  return (unsigned long long)t.x < (unsigned long long)N && (unsigned long long)t.y < (unsigned long long)N &&
         (unsigned long long)t.z < (unsigned long long)N && (unsigned long long)t.w < (unsigned long long)N;
}

// the six vertex pairs of a tet: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
__device__ __forceinline__ int pair_a(int e) { return e < 3 ? 0 : (e < 5 ? 1 : 2); }
__device__ __forceinline__ int pair_b(int e) { return e < 3 ? e + 1 : (e < 5 ? e - 1 : 3); }

// ---------------------------------------------------------------------------
// device-wide exclusive scan of int counts (N entries) into off[0..N], with
// off[N] = total; three kernels (block sums, scan of the sums, block scans)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T block_scan_excl(T v, T* total) {
  __shared__ T ws[SCAN_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = (lane < SCAN_T / 32) ? ws[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane < SCAN_T / 32) ws[lane] = s;
  }
  __syncthreads();
  const T base = (wid > 0) ? ws[wid - 1] : T(0);
  *total = ws[SCAN_T / 32 - 1];
  __syncthreads();
  return base + inc - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(const int* __restrict__ cnt, long long n,
                                                      long long* __restrict__ sums) {
  const long long b0 = (long long)blockIdx.x * SCAN_CHUNK;
  long long acc = 0;
  for (long long i = b0 + threadIdx.x; i < min(n, b0 + SCAN_CHUNK); i += SCAN_T) acc += cnt[i];
  long long tot;
  block_scan_excl<long long>(acc, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_top(long long* __restrict__ sums, int nb,
                                                     long long* total) {
  long long carry = 0;
  for (int base = 0; base < nb; base += SCAN_T) {
    const int i = base + threadIdx.x;
    const long long v = (i < nb) ? sums[i] : 0;
    long long tot;
    const long long ex = block_scan_excl<long long>(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const int* __restrict__ cnt, long long n,
                                                        const long long* __restrict__ sums,
                                                        long long* __restrict__ off) {
  const long long b0 = (long long)blockIdx.x * SCAN_CHUNK;
  constexpr int PER = SCAN_CHUNK / SCAN_T;
  const long long i0 = b0 + (long long)threadIdx.x * PER;
  int v[PER];
  long long acc = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    v[q] = (i0 + q < n) ? cnt[i0 + q] : 0;
    acc += v[q];
  }
  long long tot;
  long long run = block_scan_excl<long long>(acc, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (i0 + q < n) off[i0 + q] = run;
    run += v[q];
  }
  if (i0 <= n - 1 && n - 1 < i0 + PER) off[n] = run;   // the thread holding the last entry
}

// Returns the number of kernels launched; *total (device) receives the sum.
int scan_counts(const int* cnt, long long n, long long* sums, long long* off, long long* total,
                cudaStream_t s) {
  const int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
  k_scan_sums<<<nb, SCAN_T, 0, s>>>(cnt, n, sums);
  k_scan_top<<<1, SCAN_T, 0, s>>>(sums, nb, total);
  k_scan_blocks<<<nb, SCAN_T, 0, s>>>(cnt, n, sums, off);
  return 3;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int grid_for(long long n) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 148;
  }
  const long long b = (n + RT - 1) / RT;
  return (int)std::max<long long>(1, std::min<long long>(b, 8LL * sms));
}

// vertex and tet counts the geometry terms accept (6 K edge slots in int32)
bool sizes_ok(long long N, long long K) {
  return N >= 1 && K >= 1 && N <= 0x7fffffffLL && 6 * K <= 0x7fffffffLL;
}

}  // namespace
}  // namespace tts
