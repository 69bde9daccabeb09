// Pre-filter (Sec. 3.2), per-view preprocess and tile binning with a device
// radix sort of (tile id, mean depth) keys (Sec. 3.3).
#include <algorithm>

#include "geometry.cuh"
#include "launch.h"

namespace tts {

// ---------------------------------------------------------------------------
// block-level helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan over the block; returns the block total in *total.
template <typename T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_sums[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = (lane < NT / 32) ? warp_sums[lane] : T(0);
    s = warp_incl_scan(s);
    if (lane < NT / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const T base = (wid > 0) ? warp_sums[wid - 1] : T(0);
  *total = warp_sums[NT / 32 - 1];
  __syncthreads();
  return base + inc - v;
}

// ---------------------------------------------------------------------------
// per-call resets
// ---------------------------------------------------------------------------
__global__ void k_fwd_reset(const Batch* __restrict__ B) {
  Counters* c = B->ctr;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->zmin_bits = 0xffffffffu;
    c->zmax_bits = 0u;
    c->depth_bits = 0;
    c->total_bits = 0;
    c->n_passes = 0;
    c->n_keys = 0;
    c->n_keys_used = 0;
    c->status &= ~(unsigned)TTS_STATUS_KEY_OVERFLOW;
    c->work_fwd = c->work_bwd = 0u;
    c->done_fwd = c->done_bwd = 0u;
    c->sort_epoch += 1u;
    c->seg_total = 0;
    for (int p = 0; p < MAX_PASSES; ++p) c->sort_ticket[p] = 0u;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < B->total_tiles; t += gridDim.x * blockDim.x)
    B->ranges[t] = make_int2(0, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MAX_PASSES * RADIX; i += gridDim.x * blockDim.x)
    B->ghist[i] = 0u;
}

// ---------------------------------------------------------------------------
// K1: pre-filter.  alpha_max = Eq. 1 at (f_max, f_min) of the tet's vertices,
// keep iff alpha_max >= T_f.  Flags, then a stable compaction.
// grid (max_pf_chunks, n_scenes)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PF_THREADS) k_prefilter_flags(const Batch* __restrict__ B) {
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int chunk = blockIdx.x;
  if (chunk >= S.pf_chunks) return;
  const long long k0 = (long long)chunk * PF_CHUNK;
  const long long k1 = min(k0 + PF_CHUNK, S.K);
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float sv = B->s, thr = B->prefilter_thresh;
  // alpha_max <= sigmoid(-s f_min) < T_f once f_min > ln(1/T_f - 1)/s: such a
  // tet (most of the grid, away from the surface) needs no exponentials
  const float fcut = (thr > 0.f && thr < 1.f) ? logf(1.f / thr - 1.f) / sv : __int_as_float(0x7f800000);
  const unsigned N = (unsigned)S.N;
  unsigned char* flags = B->pf_flags + S.flag_off;
  int cnt = 0;
  bool bad = false;
#pragma unroll 4
  for (long long k = k0 + threadIdx.x; k < k1; k += PF_THREADS) {
    const int4 t = __ldg(&S.T[k]);
    unsigned char keep = 0;
    if ((unsigned)t.x < N && (unsigned)t.y < N && (unsigned)t.z < N && (unsigned)t.w < N) {
      if (pure) {
        keep = 1;
      } else {
        const float fa = __ldg(S.f + t.x), fb = __ldg(S.f + t.y), fc = __ldg(S.f + t.z),
                    fd = __ldg(S.f + t.w);
        const float fmx = fmaxf(fmaxf(fa, fb), fmaxf(fc, fd));
        const float fmn = fminf(fminf(fa, fb), fminf(fc, fd));
        // Eq. 1 at (f_max, f_min): -expm1(-s (fmax - fmin)) * sigmoid(-s fmin)
        if (fmx > fmn && fmn <= fcut) {
          const float amax = -expm1f(-sv * (fmx - fmn)) / (1.f + expf(sv * fmn));
          keep = (amax >= thr) ? 1 : 0;
        }
      }
    } else {
      bad = true;
    }
    flags[k] = keep;
    cnt += keep;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(B->ctr, TTS_STATUS_BAD_INDEX);
  int total;
  block_excl_scan<int, PF_THREADS>(cnt, &total);
  if (threadIdx.x == 0) B->pf_blocksum[S.pf_chunk_base + chunk] = total;
}

// Single block: per-scene exclusive scans of the pre-filter block counts.
__global__ void __launch_bounds__(SCAN_THREADS) k_prefilter_scan(const Batch* __restrict__ B) {
  for (int s = 0; s < B->n_scenes; ++s) {
    const SceneD& S = B->sc[s];
    int* a = B->pf_blocksum + S.pf_chunk_base;
    int carry = 0;
    for (int base = 0; base < S.pf_chunks; base += SCAN_THREADS) {
      const int i = base + threadIdx.x;
      const int v = (i < S.pf_chunks) ? a[i] : 0;
      int tot;
      const int ex = block_excl_scan<int, SCAN_THREADS>(v, &tot);
      if (i < S.pf_chunks) a[i] = carry + ex;
      carry += tot;
    }
    if (threadIdx.x == 0) {
      int n = carry;
      if ((long long)n > S.surv_cap) {
        set_status(B->ctr, TTS_STATUS_SURV_OVERFLOW);
        n = (int)S.surv_cap;
      }
      B->ctr->n_surv[s] = n;
    }
    __syncthreads();
  }
}

// Stable compaction: survivors in original tet order.
__global__ void __launch_bounds__(PF_THREADS) k_prefilter_compact(const Batch* __restrict__ B) {
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int chunk = blockIdx.x;
  if (chunk >= S.pf_chunks) return;
  constexpr int PER = PF_CHUNK / PF_THREADS;  // 16 consecutive flags per thread
  const long long k0 = (long long)chunk * PF_CHUNK + (long long)threadIdx.x * PER;
  const unsigned char* flags = B->pf_flags + S.flag_off;
  unsigned char fl[PER];
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const long long k = k0 + q;
    fl[q] = (k < S.K) ? flags[k] : 0;
    cnt += fl[q];
  }
  int total;
  int off = block_excl_scan<int, PF_THREADS>(cnt, &total) + B->pf_blocksum[S.pf_chunk_base + chunk];
  int* out = B->surv + S.surv_off;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (fl[q]) {
      if (off < S.surv_cap) out[off] = (int)(k0 + q);
      ++off;
    }
  }
}

// Per-survivor world unit normal n = g / |g| of the tet's affine SDF (Sec. 3.2
// per-tet normal, App. A.3), view independent and hoisted into the scene
// preparation (App. B.1).  grid (blocks, n_scenes)
__global__ void __launch_bounds__(256) k_tet_normals(const Batch* __restrict__ B) {
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int nsurv = B->ctr->n_surv[s];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nsurv; k += gridDim.x * blockDim.x) {
    const int4 t = __ldg(&S.T[B->surv[S.surv_off + k]]);
    const int id[4] = {t.x, t.y, t.z, t.w};
    float3 v[4];
    float f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float* p = S.V + 3ll * id[j];
      v[j] = f3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
      f[j] = __ldg(S.f + id[j]);
    }
    TetGrad G;
    tet_grad(v, f, G);
    float ih, sg;
    const float3 n = tet_unit_normal(G, &ih, &sg);
    B->surv_n[S.surv_off + k] = make_float4(n.x, n.y, n.z, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Coarse-to-fine pre-filter (App. B.1): the axis-aligned bounds of the
// survivors' vertices after a first round, and the affine refit of the grid
// into those bounds for the second round.  Float min / max go through
// order-preserving unsigned keys so that plain integer atomics apply.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned float_key(float x) {
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_bounds_init(const Batch* __restrict__ B) {
  const int i = threadIdx.x;
  if (i < 6 * B->n_scenes) B->bounds[i] = (i % 6 < 3) ? 0xffffffffu : 0u;
}

// grid (blocks, n_scenes)
__global__ void __launch_bounds__(256) k_bounds(const Batch* __restrict__ B) {
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int nsurv = B->ctr->n_surv[s];
  unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nsurv; k += gridDim.x * blockDim.x) {
    const int4 t = __ldg(&S.T[B->surv[S.surv_off + k]]);
    const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const unsigned key = float_key(__ldg(S.V + 3ll * id[j] + r));
        mn[r] = min(mn[r], key);
        mx[r] = max(mx[r], key);
      }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    mn[r] = __reduce_min_sync(0xffffffffu, mn[r]);
    mx[r] = __reduce_max_sync(0xffffffffu, mx[r]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (mn[r] != 0xffffffffu) atomicMin(&B->bounds[6 * s + r], mn[r]);
      if (mx[r] != 0u) atomicMax(&B->bounds[6 * s + 3 + r], mx[r]);
    }
  }
}

// empty scenes read back as (+inf, +inf, +inf, -inf, -inf, -inf)
__global__ void k_bounds_finish(const Batch* __restrict__ B, float* __restrict__ aabb) {
  const int i = threadIdx.x;
  if (i >= 6 * B->n_scenes) return;
  const unsigned k = B->bounds[i];
  const bool empty = (i % 6 < 3) ? (k == 0xffffffffu) : (k == 0u);
  aabb[i] = empty ? ((i % 6 < 3) ? __int_as_float(0x7f800000) : __int_as_float(0xff800000))
                  : key_float(k);
}

int launch_bounds(const HostPlan& P, const Batch* dB, float* aabb, cudaStream_t st) {
  k_bounds_init<<<1, 6 * TTS_MAX_SCENES, 0, st>>>(dB);
  k_bounds<<<dim3(P.normal_blocks, P.n_scenes), 256, 0, st>>>(dB);
  k_bounds_finish<<<1, 6 * TTS_MAX_SCENES, 0, st>>>(dB, aabb);
  return 3;
}

struct FitArgs {
  float lo[3], hi[3];
};

// V_out = b_lo + (V_in - lo) * (b_hi - b_lo) / (hi - lo) per axis, [b_lo, b_hi]
// the bounds widened by pad * extent on each side; unchanged when empty.
__global__ void __launch_bounds__(256) k_fit_grid(const float* __restrict__ Vin, long long N,
                                                  FitArgs a, const float* __restrict__ aabb,
                                                  float pad, float* __restrict__ Vout) {
  float scale[3], off[3];
  bool empty = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) empty |= !(aabb[r] <= aabb[3 + r]);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float ext = aabb[3 + r] - aabb[r];
    const float blo = aabb[r] - pad * ext, bhi = aabb[3 + r] + pad * ext;
    scale[r] = empty ? 1.f : (bhi - blo) / (a.hi[r] - a.lo[r]);
    off[r] = empty ? 0.f : blo - a.lo[r] * scale[r];
  }
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < 3 * N; i += (long long)gridDim.x * 256) {
    const int r = (int)(i % 3);
    Vout[i] = __fmaf_rn(Vin[i], scale[r], off[r]);
  }
}

int launch_fit_grid(const float* V_in, long long N, const float lo[3], const float hi[3],
                    const float* aabb, float pad, float* V_out, cudaStream_t st) {
  FitArgs a;
  for (int r = 0; r < 3; ++r) {
    a.lo[r] = lo[r];
    a.hi[r] = hi[r];
  }
  const long long blocks = std::min<long long>((3 * N + 255) / 256, 4096);
  k_fit_grid<<<(int)blocks, 256, 0, st>>>(V_in, N, a, aabb, pad, V_out);
  return 1;
}

// ---------------------------------------------------------------------------
// K2: per-view preprocess.  grid (max_pp_chunks, n_views)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PP_THREADS, 3) k_preprocess(const Batch* __restrict__ B) {
  const int v = blockIdx.y;
  const ViewD& vw = B->vw[v];
  const int chunk = blockIdx.x;
  if (chunk >= vw.pp_chunks) return;
  const SceneD& S = B->sc[vw.scene];
  const int nsurv = B->ctr->n_surv[vw.scene];
  const float s = B->s;
  const int tile = B->tile;
  long long nt_sum = 0;
  unsigned zmn = 0xffffffffu, zmx = 0u;
  for (int q = threadIdx.x; q < PP_CHUNK; q += PP_THREADS) {
    const int k = chunk * PP_CHUNK + q;
    if (k >= nsurv) break;
    const long long slot = vw.rec_base + k;
    const int tet = B->surv[S.surv_off + k];
    TetIn in;
    load_tet(S, tet, in);
    Geo G;
    tet_geometry(vw, s, in, G);
    int nt = 0;
    if (G.visible) {
      const int tx0 = G.i0 / tile, tx1 = G.i1 / tile, ty0 = G.j0 / tile, ty1 = G.j1 / tile;
      nt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
      B->rec_rect[slot] = make_int4(tx0, tx1, ty0, ty1);
      write_record(vw, s, in, G, B->rec + slot * REC_Q);
      zmn = min(zmn, G.zbits);
      zmx = max(zmx, G.zbits);
    }
    B->rec_nt[slot] = nt;
    B->rec_z[slot] = G.zbits;
    nt_sum += nt;
  }
  long long tot;
  block_excl_scan<long long, PP_THREADS>(nt_sum, &tot);
  // block min/max of the depth bits
  __shared__ unsigned smn, smx;
  if (threadIdx.x == 0) { smn = 0xffffffffu; smx = 0u; }
  __syncthreads();
  if (zmn != 0xffffffffu) { atomicMin(&smn, zmn); atomicMax(&smx, zmx); }
  __syncthreads();
  if (threadIdx.x == 0) {
    B->pp_blocksum[vw.pp_chunk_base + chunk] = tot;
    if (smn != 0xffffffffu) {
      atomicMin(&B->ctr->zmin_bits, smn);
      atomicMax(&B->ctr->zmax_bits, smx);
    }
  }
}

// Single block: exclusive scan of all preprocess block sums (views in order)
// -> key offsets; total -> n_keys; key encoding bit counts.
__global__ void __launch_bounds__(SCAN_THREADS) k_preprocess_scan(const Batch* __restrict__ B) {
  long long* a = B->pp_blocksum;
  const int n = B->pp_chunks_total;
  long long carry = 0;
  for (int base = 0; base < n; base += SCAN_THREADS) {
    const int i = base + threadIdx.x;
    const long long v = (i < n) ? a[i] : 0;
    long long tot;
    const long long ex = block_excl_scan<long long, SCAN_THREADS>(v, &tot);
    if (i < n) a[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    Counters* c = B->ctr;
    c->n_keys = carry;
    long long used = carry;
    if (carry > B->key_cap) {
      set_status(c, TTS_STATUS_KEY_OVERFLOW);
      used = 0;
    }
    c->n_keys_used = used;
    unsigned span = (c->zmax_bits >= c->zmin_bits) ? (c->zmax_bits - c->zmin_bits) : 0u;
    if (c->zmin_bits == 0xffffffffu) span = 0;
    const int db = (span == 0) ? 0 : (32 - __clz(span));
    c->depth_bits = db;
    c->total_bits = db + B->tile_bits;
    c->n_passes = (used > 1) ? (c->total_bits + RADIX_BITS - 1) / RADIX_BITS : 0;
  }
}

// ---------------------------------------------------------------------------
// K3: duplicate.  One key per (slot, overlapped tile), in slot order and
// row-major tile order within the slot's rect.  grid (max_pp_chunks, n_views)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PP_THREADS) k_duplicate(const Batch* __restrict__ B) {
  const int v = blockIdx.y;
  const ViewD& vw = B->vw[v];
  const int chunk = blockIdx.x;
  if (chunk >= vw.pp_chunks) return;
  const Counters* c = B->ctr;
  if (c->n_keys_used == 0) return;
  const int nsurv = c->n_surv[vw.scene];
  constexpr int PER = PP_CHUNK / PP_THREADS;
  // thread handles PER consecutive slots so that key order follows slot order
  const int k0 = chunk * PP_CHUNK + threadIdx.x * PER;
  int nt[PER];
  long long cnt = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int k = k0 + q;
    nt[q] = (k < nsurv) ? B->rec_nt[vw.rec_base + k] : 0;
    cnt += nt[q];
  }
  long long tot;
  long long off = block_excl_scan<long long, PP_THREADS>(cnt, &tot) + B->pp_blocksum[vw.pp_chunk_base + chunk];
  const unsigned zmin = c->zmin_bits;
  const int db = c->depth_bits;
  unsigned long long* keys = B->keys[0];
  unsigned int* vals = B->vals[0];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (nt[q] == 0) continue;
    const long long slot = vw.rec_base + k0 + q;
    const int4 r = B->rec_rect[slot];
    const unsigned long long zrel = (unsigned long long)(B->rec_z[slot] - zmin);
    for (int ty = r.z; ty <= r.w; ++ty)
      for (int tx = r.x; tx <= r.y; ++tx) {
        const unsigned long long gt = (unsigned long long)(vw.tile_base + ty * vw.tiles_x + tx);
        keys[off] = (gt << db) | zrel;
        vals[off] = (unsigned)slot;
        ++off;
      }
  }
}

// ---------------------------------------------------------------------------
// K4: LSD radix sort, 8-bit digits, stable, one kernel per digit pass.  The
// global digit counts of every pass come from one read of the keys
// (k_radix_ghist).  A pass takes tiles of SORT_TILE keys in ticket order,
// ranks them per digit inside the block (warp multisplit), publishes the
// tile's digit counts, finds the counts of all earlier tiles by decoupled
// look-back (each earlier tile's aggregate, or the inclusive prefix where one
// is published), publishes its own inclusive prefix and scatters the tile in
// digit runs.  The look-back waits are bounded: past the limit the pass sets
// TTS_STATUS_TIMEOUT and goes on (its output is then undefined).
// ---------------------------------------------------------------------------
constexpr unsigned long long LB_AGG = 1ull << 32;      // flag bits above the 32-bit count
constexpr unsigned long long LB_PREFIX = 2ull << 32;
constexpr long long LB_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ unsigned long long lb_word(unsigned tag, unsigned long long flag,
                                                      unsigned value) {
  return ((unsigned long long)tag << 34) | flag | value;
}

// grid: sort_blocks; each block adds its keys' digits of every live pass
__global__ void __launch_bounds__(SORT_THREADS) k_radix_ghist(const Batch* __restrict__ B) {
  const Counters* c = B->ctr;
  const int np = c->n_passes;
  if (np == 0) return;
  const long long n = c->n_keys_used;
  constexpr int NH = SORT_THREADS / 64;   // one histogram per two warps (32 KB)
  __shared__ unsigned h[NH][MAX_PASSES][RADIX];
  for (int i = threadIdx.x; i < NH * MAX_PASSES * RADIX; i += SORT_THREADS) (&h[0][0][0])[i] = 0;
  __syncthreads();
  const unsigned long long* src = B->keys[0];
  const int wid = threadIdx.x >> 6;
  for (long long i = blockIdx.x * (long long)SORT_THREADS + threadIdx.x; i < n;
       i += (long long)gridDim.x * SORT_THREADS) {
    const unsigned long long k = src[i];
    for (int p = 0; p < np; ++p) atomicAdd(&h[wid][p][(unsigned)(k >> (p * RADIX_BITS)) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < np * RADIX; i += SORT_THREADS) {
    unsigned t = 0;
#pragma unroll
    for (int w = 0; w < NH; ++w) t += (&h[w][0][0])[i];
    if (t) atomicAdd(&B->ghist[i], t);
  }
}

// grid: sort_tiles (the key capacity's tiles); blocks past the live tiles exit
__global__ void __launch_bounds__(SORT_THREADS) k_radix_onesweep(const Batch* __restrict__ B, int pass) {
  Counters* c = B->ctr;
  if (pass >= c->n_passes) return;
  const long long n = c->n_keys_used;
  const int ntiles = (int)((n + SORT_TILE - 1) / SORT_TILE);
  constexpr int NW = SORT_THREADS / 32;
  __shared__ int s_tile;
  __shared__ unsigned dbase[RADIX];
  __shared__ unsigned wcnt[NW][RADIX];
  __shared__ unsigned tstart[RADIX];
  __shared__ unsigned long long sk[SORT_TILE];
  __shared__ unsigned sv[SORT_TILE];
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(&c->sort_ticket[pass], 1u);
  for (int i = threadIdx.x; i < NW * RADIX; i += SORT_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int tile = s_tile;
  if (tile >= ntiles) return;
  const unsigned tag = (c->sort_epoch * MAX_PASSES + pass) % 0xffffu + 1u;
  const long long t0 = (long long)tile * SORT_TILE;
  const int tn = (int)min((long long)SORT_TILE, n - t0);
  const unsigned long long* ksrc = B->keys[pass & 1];
  const unsigned* vsrc = B->vals[pass & 1];
  unsigned long long* kdst = B->keys[(pass + 1) & 1];
  unsigned* vdst = B->vals[(pass + 1) & 1];
  const int sh = pass * RADIX_BITS;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long k[SORT_KPT];
  unsigned val[SORT_KPT], dg[SORT_KPT], off[SORT_KPT];
#pragma unroll
  for (int j = 0; j < SORT_KPT; ++j) {
    const int i = wid * (32 * SORT_KPT) + j * 32 + lane;
    if (i < tn) {
      k[j] = ksrc[t0 + i];
      val[j] = vsrc[t0 + i];
      dg[j] = (unsigned)(k[j] >> sh) & (RADIX - 1);
    } else {
      dg[j] = RADIX;  // sentinel: not scattered
    }
  }
  // ranks inside each warp (warp multisplit), digit counts per warp
#pragma unroll
  for (int j = 0; j < SORT_KPT; ++j) {
    const unsigned peers = __match_any_sync(0xffffffffu, dg[j]);
    const unsigned rank = __popc(peers & lt_mask);
    const unsigned d = dg[j] & (RADIX - 1);
    const unsigned before = (dg[j] < RADIX) ? wcnt[wid][d] : 0u;
    __syncwarp();
    if (dg[j] < RADIX && rank == 0) wcnt[wid][d] = before + __popc(peers);
    __syncwarp();
    off[j] = before + rank;
  }
  __syncthreads();
  {
    const int d = threadIdx.x;   // SORT_THREADS == RADIX
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const unsigned x = wcnt[w][d];
      wcnt[w][d] = run;
      run += x;
    }
    unsigned t;
    tstart[d] = block_excl_scan<unsigned, SORT_THREADS>(run, &t);
    // publish this tile's count of digit d, then look back over the earlier
    // tiles for their counts
    unsigned long long* look = B->look + (size_t)tile * RADIX + d;
    if (tile > 0) atomicExch(look, lb_word(tag, LB_AGG, run));
    unsigned excl = 0;
    bool timed_out = false;
    for (int tp = tile - 1; tp >= 0;) {
      const unsigned long long w =
          *reinterpret_cast<volatile unsigned long long*>(B->look + (size_t)tp * RADIX + d);
      if ((unsigned)(w >> 34) == tag && (w & (LB_AGG | LB_PREFIX))) {
        excl += (unsigned)w;
        if (w & LB_PREFIX) break;
        --tp;
        continue;
      }
      long long spins = 0;
      while (true) {   // the earlier tile has not published yet: bounded wait
        const unsigned long long w2 =
            *reinterpret_cast<volatile unsigned long long*>(B->look + (size_t)tp * RADIX + d);
        if ((unsigned)(w2 >> 34) == tag && (w2 & (LB_AGG | LB_PREFIX))) break;
        if (++spins > LB_SPIN_LIMIT) {
          timed_out = true;
          break;
        }
      }
      if (timed_out) break;
    }
    if (timed_out) set_status(c, TTS_STATUS_TIMEOUT);
    atomicExch(look, lb_word(tag, LB_PREFIX, excl + run));
    // digit base: all smaller digits of the whole pass, then the earlier tiles
    const unsigned g = B->ghist[pass * RADIX + d];
    unsigned tg;
    dbase[d] = block_excl_scan<unsigned, SORT_THREADS>(g, &tg) + excl;
  }
  __syncthreads();
  // stage the tile in digit order, then write each digit's run contiguously
#pragma unroll
  for (int j = 0; j < SORT_KPT; ++j) {
    if (dg[j] < RADIX) {
      const unsigned lp = tstart[dg[j]] + wcnt[wid][dg[j]] + off[j];
      sk[lp] = k[j];
      sv[lp] = val[j];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < tn; q += SORT_THREADS) {
    const unsigned long long key = sk[q];
    const unsigned d = (unsigned)(key >> sh) & (RADIX - 1);
    const unsigned pos = dbase[d] + (unsigned)q - tstart[d];
    kdst[pos] = key;
    vdst[pos] = sv[q];
  }
}

// K5: per-tile [start, end) from the sorted keys.
__global__ void k_tile_ranges(const Batch* __restrict__ B) {
  const Counters* c = B->ctr;
  const long long n = c->n_keys_used;
  const int db = c->depth_bits;
  const unsigned long long* keys = B->keys[c->n_passes & 1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(keys[i] >> db);
    if (i == 0 || (int)(keys[i - 1] >> db) != t) B->ranges[t].x = (int)i;
    if (i == n - 1 || (int)(keys[i + 1] >> db) != t) B->ranges[t].y = (int)(i + 1);
  }
}

// Work list for the persistent blend kernels, units (tile, segment | part << 24).
// A tile whose list is longer than seg_len entries is split into segments of
// seg_len entries: the forward walks the whole list (the segment-0 units,
// parts 0 and 1 covering its 4x4 blocks) and records its state at each
// segment end, and the backward walks the segments in parallel from those
// states (one warp per 8x4 block walking a long list back to front would
// otherwise bound its duration).  Units (tile, segment) are ordered by
// decreasing work (bucketed by bit length), so the longest start first; the
// order inside a bucket is arbitrary.
// Warp-level exclusive scan of v (all lanes), returning the warp total.
__device__ __forceinline__ int warp_excl_scan(int v, int* total) {
  const int lane = threadIdx.x & 31;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  *total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - v;
}

constexpr int WL_BUCKETS = 34;      // bit length of a work amount (0..32), 33: unused
constexpr int WL_THREADS = 256;     // one tile per thread

// Work-list step 1 (one tile per thread): segment count and checkpoint slots
// of each tile, and per block the units of each length bucket.
__global__ void __launch_bounds__(WL_THREADS) k_worklist_count(const Batch* __restrict__ B) {
  __shared__ int cnt[WL_BUCKETS];
  if (threadIdx.x < WL_BUCKETS) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int t = blockIdx.x * WL_THREADS + threadIdx.x;
  const int nt = B->total_tiles;
  const int L = B->seg_len;
  const int lane = threadIdx.x & 31;
  const bool in = t < nt;
  const int2 r = in ? B->ranges[t] : make_int2(0, 0);
  const int len = r.y - r.x;
  int nseg = (in && L > 0 && len > L) ? (len + L - 1) / L : 1;
  // checkpoint slots, one atomic per warp
  int tot;
  const int ex = warp_excl_scan(nseg > 1 ? nseg : 0, &tot);
  int base0 = 0;
  if (lane == 31 && tot > 0) base0 = atomicAdd(&B->ctr->seg_total, tot);
  base0 = __shfl_sync(0xffffffffu, base0, 31);
  int base = -1;
  if (nseg > 1) {
    base = base0 + ex;
    if (base + nseg > B->seg_cap) {   // outside the sizing bound: blend unsplit
      nseg = 1;
      base = -1;
    }
  }
  if (in) {
    B->tseg[t] = make_int2(base, nseg);
    // segment 0 carries the forward's walk of the whole list (two parts for
    // a split list): bucketed by the list length; the later segments
    // (backward only) by the segment length
    atomicAdd(&cnt[len > 0 ? 32 - __clz(len) : 0], nseg > 1 ? 2 : 1);
    if (nseg > 1) atomicAdd(&cnt[32 - __clz(L)], nseg - 1);
  }
  __syncthreads();
  if (threadIdx.x < WL_BUCKETS) B->wl_blockcnt[blockIdx.x * WL_BUCKETS + threadIdx.x] = cnt[threadIdx.x];
}

// Work-list step 2 (one block of 17 warps, two buckets each): per bucket,
// the exclusive prefix of the blocks' unit counts (in place) and, over the
// buckets from the longest down, the first unit of each bucket.
__global__ void __launch_bounds__(17 * 32) k_worklist_scan(const Batch* __restrict__ B, int nb) {
  __shared__ int total[WL_BUCKETS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j < WL_BUCKETS; j += 17) {
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
      const int b = b0 + lane;
      const int v = (b < nb) ? B->wl_blockcnt[b * WL_BUCKETS + j] : 0;
      int tot;
      const int ex = warp_excl_scan(v, &tot);
      if (b < nb) B->wl_blockcnt[b * WL_BUCKETS + j] = carry + ex;
      carry += tot;
    }
    if (lane == 0) total[j] = carry;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int j = WL_BUCKETS - 1; j >= 0; --j) {
      B->wl_base[j] = run;
      run += total[j];
    }
    B->ctr->n_units = run;
  }
}

// Work-list step 3 (one tile per thread): each tile's units go after all
// units of longer buckets and after the earlier blocks' units of its bucket.
__global__ void __launch_bounds__(WL_THREADS) k_worklist_place(const Batch* __restrict__ B) {
  __shared__ int off[WL_BUCKETS];
  if (threadIdx.x < WL_BUCKETS)
    off[threadIdx.x] = B->wl_base[threadIdx.x] + B->wl_blockcnt[blockIdx.x * WL_BUCKETS + threadIdx.x];
  __syncthreads();
  const int t = blockIdx.x * WL_THREADS + threadIdx.x;
  if (t >= B->total_tiles) return;
  const int L = B->seg_len;
  const int2 r = B->ranges[t];
  const int2 ts = B->tseg[t];
  const int len = r.y - r.x;
  const int pos0 = atomicAdd(&off[len > 0 ? 32 - __clz(len) : 0], ts.y > 1 ? 2 : 1);
  B->worklist[pos0] = make_int2(t, 0);
  if (ts.y > 1) {
    B->worklist[pos0 + 1] = make_int2(t, 1 << 24);   // part 1: forward only
    const int pos = atomicAdd(&off[32 - __clz(L)], ts.y - 1);
    for (int j = 1; j < ts.y; ++j) B->worklist[pos + j - 1] = make_int2(t, j);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_prefilter(const HostPlan& P, const Batch* dB, cudaStream_t st) {
  dim3 g(P.max_pf_chunks, P.n_scenes);
  k_prefilter_flags<<<g, PF_THREADS, 0, st>>>(dB);
  k_prefilter_scan<<<1, SCAN_THREADS, 0, st>>>(dB);
  k_prefilter_compact<<<g, PF_THREADS, 0, st>>>(dB);
  if (P.normals) {
    k_tet_normals<<<dim3(P.normal_blocks, P.n_scenes), 256, 0, st>>>(dB);
    return 4;
  }
  return 3;
}

int launch_binning(const HostPlan& P, const Batch* dB, cudaStream_t st) {
  k_fwd_reset<<<64, 256, 0, st>>>(dB);
  dim3 g(P.max_pp_chunks, P.n_views);
  k_preprocess<<<g, PP_THREADS, 0, st>>>(dB);
  k_preprocess_scan<<<1, SCAN_THREADS, 0, st>>>(dB);
  k_duplicate<<<g, PP_THREADS, 0, st>>>(dB);
  k_radix_ghist<<<P.sort_blocks, SORT_THREADS, 0, st>>>(dB);
  for (int p = 0; p < P.max_passes; ++p) {
    k_radix_onesweep<<<P.sort_tiles, SORT_THREADS, 0, st>>>(dB, p);
  }
  k_tile_ranges<<<P.range_blocks, 256, 0, st>>>(dB);
  k_worklist_count<<<P.wl_blocks, WL_THREADS, 0, st>>>(dB);
  k_worklist_scan<<<1, 17 * 32, 0, st>>>(dB, P.wl_blocks);
  k_worklist_place<<<P.wl_blocks, WL_THREADS, 0, st>>>(dB);
  return 9 + P.max_passes;
}

}  // namespace tts
