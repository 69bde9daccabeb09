// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits,
// three kernels per pass (per-block digit counts, a scan of each digit's row
// over the blocks, a stable scatter ranked per warp by match_any).  Only the
// low key_bits bits of a key take part in the order: the last pass reads a
// digit of key_bits - 8 (passes - 1) bits.  Two entry points: tts_sort_pairs
// sorts in caller-provided scratch; tts_sort_pairs_noalloc sorts in a scratch
// array compiled into the library.
//
// tts_sort_pairs_noalloc:
// Who needs it: callers that must not allocate device memory themselves, for
// example a custom allocator hook (which cannot call back into cudaMalloc),
// plugin hosts that own every device allocation, or latency-critical loops
// that cannot afford cudaMalloc's implicit device synchronisation.  They pass
// inputs and outputs; the temporary storage lives in a fixed-size array
// compiled into this file.
//
// Limits and sharing rules:
//  * at most TTS_SORT_NOALLOC_MAX_KEYS pairs per call; larger calls return
//    TTS_ERR_ARG before anything is enqueued;
//  * the scratch array (about 12.3 MiB) exists on every device that loads the
//    library, until the process exits;
//  * all calls on a device share it: calls whose work overlaps on the GPU
//    (different streams without ordering between them) race and corrupt each
//    other's results;
//  * the first call on a device looks up the array's device address (a
//    cudaGetSymbolAddress call); make that first call before any stream
//    capture on that device.
// Nothing in the scratch needs to start at zero: every pass rewrites the
// histogram rows it reads.
//
// Errors: each kernel is launched with cudaLaunchKernelEx and its own return
// code is checked, so an error left pending by unrelated earlier CUDA calls
// is neither reported as this call's nor cleared.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "tets.h"

namespace tts {
void count_launches(long long n);
}

namespace {

constexpr int NA_RADIX = 256;
constexpr int NA_THREADS = 256;
constexpr int NA_KPT = 8;
constexpr int NA_TILE = NA_THREADS * NA_KPT;
constexpr int NA_BLOCKS = 256;
constexpr long long NA_MAX_KEYS = TTS_SORT_NOALLOC_MAX_KEYS;

struct NaScratch {
  unsigned long long keys[NA_MAX_KEYS];
  unsigned int vals[NA_MAX_KEYS];
  unsigned int hist[NA_RADIX * (NA_BLOCKS + 1)];
};

static __device__ __align__(256) NaScratch g_na_scratch;

__device__ __forceinline__ void na_chunk(long long n, long long* lo, long long* hi) {
  long long per = (n + NA_BLOCKS - 1) / NA_BLOCKS;
  per = (per + NA_TILE - 1) / NA_TILE * NA_TILE;
  *lo = min(n, per * blockIdx.x);
  *hi = min(n, *lo + per);
}

template <typename T>
__device__ __forceinline__ T na_block_excl_scan(T v, T* total) {
  __shared__ T ws[NA_THREADS / 32];
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
    T s = (lane < NA_THREADS / 32) ? ws[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane < NA_THREADS / 32) ws[lane] = s;
  }
  __syncthreads();
  const T base = (wid > 0) ? ws[wid - 1] : T(0);
  *total = ws[NA_THREADS / 32 - 1];
  __syncthreads();
  return base + inc - v;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_hist(const unsigned long long* __restrict__ src,
                                                        long long n, int shift, unsigned mask,
                                                        unsigned* __restrict__ hist) {
  long long lo, hi;
  na_chunk(n, &lo, &hi);
  __shared__ unsigned h[NA_THREADS / 32][NA_RADIX];
  for (int i = threadIdx.x; i < (NA_THREADS / 32) * NA_RADIX; i += NA_THREADS) (&h[0][0])[i] = 0;
  __syncthreads();
  const int wid = threadIdx.x >> 5;
  for (long long i = lo + threadIdx.x; i < hi; i += NA_THREADS)
    atomicAdd(&h[wid][(unsigned)(src[i] >> shift) & mask], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < NA_RADIX; d += NA_THREADS) {
    unsigned t = 0;
#pragma unroll
    for (int w = 0; w < NA_THREADS / 32; ++w) t += h[w][d];
    hist[(size_t)d * (NA_BLOCKS + 1) + blockIdx.x] = t;
  }
}

// one block per digit: exclusive scan of the row over the blocks, total last
__global__ void __launch_bounds__(NA_THREADS) k_na_rowscan(unsigned* __restrict__ hist) {
  unsigned* row = hist + (size_t)blockIdx.x * (NA_BLOCKS + 1);
  unsigned carry = 0;
  for (int base = 0; base < NA_BLOCKS; base += NA_THREADS) {
    const int i = base + threadIdx.x;
    const unsigned v = (i < NA_BLOCKS) ? row[i] : 0u;
    unsigned tot;
    const unsigned ex = na_block_excl_scan<unsigned>(v, &tot);
    if (i < NA_BLOCKS) row[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) row[NA_BLOCKS] = carry;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_scatter(
    const unsigned long long* __restrict__ ksrc, const unsigned* __restrict__ vsrc,
    unsigned long long* __restrict__ kdst, unsigned* __restrict__ vdst, long long n, int shift,
    unsigned mask, const unsigned* __restrict__ hist) {
  long long lo, hi;
  na_chunk(n, &lo, &hi);
  constexpr int NW = NA_THREADS / 32;
  __shared__ unsigned base[NA_RADIX];
  __shared__ unsigned wcnt[NW][NA_RADIX];
  __shared__ unsigned tcnt[NA_RADIX];
  {
    const int d = threadIdx.x;
    unsigned t;
    const unsigned ex = na_block_excl_scan<unsigned>(hist[(size_t)d * (NA_BLOCKS + 1) + NA_BLOCKS], &t);
    base[d] = ex + hist[(size_t)d * (NA_BLOCKS + 1) + blockIdx.x];
  }
  for (int i = threadIdx.x; i < NW * NA_RADIX; i += NA_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (long long t0 = lo; t0 < hi; t0 += NA_TILE) {
    unsigned long long k[NA_KPT];
    unsigned val[NA_KPT], dg[NA_KPT], off[NA_KPT];
#pragma unroll
    for (int j = 0; j < NA_KPT; ++j) {
      const long long i = t0 + (long long)wid * (32 * NA_KPT) + j * 32 + lane;
      if (i < hi) {
        k[j] = ksrc[i];
        val[j] = vsrc[i];
        dg[j] = (unsigned)(k[j] >> shift) & mask;
      } else {
        dg[j] = NA_RADIX;
      }
    }
#pragma unroll
    for (int j = 0; j < NA_KPT; ++j) {
      const unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
      const unsigned rank = __popc(peers & lt_mask);
      const unsigned d = dg[j] & (NA_RADIX - 1);
      const unsigned before = (dg[j] < NA_RADIX) ? wcnt[wid][d] : 0u;
      __syncwarp();
      if (dg[j] < NA_RADIX && rank == 0) wcnt[wid][d] = before + __popc(peers);
      __syncwarp();
      off[j] = before + rank;
    }
    __syncthreads();
    {
      const int d = threadIdx.x;
      unsigned run = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const unsigned x = wcnt[w][d];
        wcnt[w][d] = run;
        run += x;
      }
      tcnt[d] = run;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NA_KPT; ++j) {
      if (dg[j] < NA_RADIX) {
        const unsigned pos = base[dg[j]] + wcnt[wid][dg[j]] + off[j];
        kdst[pos] = k[j];
        vdst[pos] = val[j];
      }
    }
    __syncthreads();
    {
      const int d = threadIdx.x;
      base[d] += tcnt[d];
#pragma unroll
      for (int w = 0; w < NW; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
  }
}

// Launches one kernel of the sort and returns its own launch status.
template <typename... KArgs, typename... Args>
cudaError_t na_launch(void (*kernel)(KArgs...), int grid, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NA_THREADS);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The passes over the low key_bits bits: ks/vs in, the final pass into
// kout/vout, the others into tk/tv (ping-pong), hist: NA_RADIX x (NA_BLOCKS+1).
// Pass p sorts by bits [8p, 8p + 8) masked to key_bits.  Returns TTS_OK or
// TTS_ERR_CUDA when one of its launches failed (nothing after it is enqueued).
int radix_sort_pairs(const unsigned long long* ks, const unsigned* vs, unsigned long long* kout,
                     unsigned* vout, unsigned long long* tk, unsigned* tv, unsigned* hist,
                     long long n, int key_bits, cudaStream_t st) {
  const int passes = (key_bits + 7) / 8;
  long long launched = 0;
  int rc = TTS_OK;
  for (int p = 0; p < passes && rc == TTS_OK; ++p) {
    // the pass that writes the final result targets the caller's output
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    unsigned long long* kd = to_out ? kout : tk;
    unsigned* vd = to_out ? vout : tv;
    const int bits = key_bits - 8 * p < 8 ? key_bits - 8 * p : 8;
    const unsigned mask = (1u << bits) - 1u;
    cudaError_t e = na_launch(k_na_hist, NA_BLOCKS, st, ks, n, 8 * p, mask, hist);
    if (e == cudaSuccess) { ++launched; e = na_launch(k_na_rowscan, NA_RADIX, st, hist); }
    if (e == cudaSuccess) {
      ++launched;
      e = na_launch(k_na_scatter, NA_BLOCKS, st, ks, vs, kd, vd, n, 8 * p, mask,
                    (const unsigned*)hist);
    }
    if (e == cudaSuccess) ++launched; else rc = TTS_ERR_CUDA;
    ks = kd;
    vs = vd;
  }
  tts::count_launches(launched);
  return rc;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Per-device address of the scratch array, looked up once per device (with
// that device current) and reused.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
NaScratch* g_na_ptr[NA_MAX_DEVICES] = {};

int na_scratch(NaScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return TTS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || p == nullptr) return TTS_ERR_CUDA;
    g_na_ptr[dev] = static_cast<NaScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return TTS_OK;
}

}  // namespace

extern "C" int tts_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in,
                                      uint64_t* keys_out, uint32_t* vals_out, int64_t n,
                                      int32_t key_bits, tts_stream stream) {
  if (n < 0 || n > NA_MAX_KEYS) return TTS_ERR_ARG;
  if (key_bits < 1 || key_bits > 64) return TTS_ERR_ARG;
  if (n == 0) return TTS_OK;
  if (!keys_in || !vals_in || !keys_out || !vals_out) return TTS_ERR_ARG;
  if ((const void*)keys_in == (void*)keys_out || (const void*)vals_in == (void*)vals_out)
    return TTS_ERR_ARG;
  NaScratch* S = nullptr;
  int rc = na_scratch(&S);
  if (rc != TTS_OK) return rc;
  return radix_sort_pairs(reinterpret_cast<const unsigned long long*>(keys_in), vals_in,
                          reinterpret_cast<unsigned long long*>(keys_out), vals_out, S->keys,
                          S->vals, S->hist, n, key_bits, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int tts_sort_pairs_scratch_size(int64_t n, size_t* bytes) {
  if (!bytes || n < 0 || n > 0x7fffffffLL) return TTS_ERR_ARG;
  *bytes = align256(sizeof(unsigned long long) * (size_t)n) + align256(sizeof(unsigned) * (size_t)n) +
           align256(sizeof(unsigned) * NA_RADIX * (NA_BLOCKS + 1));
  return TTS_OK;
}

extern "C" int tts_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                              uint32_t* vals_out, int64_t n, int32_t key_bits, void* scratch,
                              size_t scratch_bytes, tts_stream stream) {
  size_t need = 0;
  if (tts_sort_pairs_scratch_size(n, &need) != TTS_OK) return TTS_ERR_ARG;
  if (key_bits < 1 || key_bits > 64) return TTS_ERR_ARG;
  if (n == 0) return TTS_OK;
  if (!keys_in || !vals_in || !keys_out || !vals_out) return TTS_ERR_ARG;
  if ((const void*)keys_in == (void*)keys_out || (const void*)vals_in == (void*)vals_out)
    return TTS_ERR_ARG;
  if (!scratch || reinterpret_cast<uintptr_t>(scratch) % 256 != 0 || scratch_bytes < need)
    return TTS_ERR_WORKSPACE;
  char* base = static_cast<char*>(scratch);
  unsigned long long* tk = reinterpret_cast<unsigned long long*>(base);
  base += align256(sizeof(unsigned long long) * (size_t)n);
  unsigned* tv = reinterpret_cast<unsigned*>(base);
  base += align256(sizeof(unsigned) * (size_t)n);
  unsigned* hist = reinterpret_cast<unsigned*>(base);
  return radix_sort_pairs(reinterpret_cast<const unsigned long long*>(keys_in), vals_in,
                          reinterpret_cast<unsigned long long*>(keys_out), vals_out, tk, tv, hist,
                          n, key_bits, reinterpret_cast<cudaStream_t>(stream));
}
