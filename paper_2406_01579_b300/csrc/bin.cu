// Pre-filter (Sec. 3.2), per-view preprocess and tile binning (Sec. 3.3): keys
// bucketed by tile, then each tile's list sorted by mean depth on chip.
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

// ---------------------------------------------------------------------------
// per-call resets
// ---------------------------------------------------------------------------
__global__ void k_fwd_reset(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  Counters* c = B->ctr;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->zmin_bits = 0xffffffffu;
    c->zmax_bits = 0u;
    c->depth_bits = 0;
    c->total_bits = 0;
    c->long_lists = 0;
    c->n_keys = 0;
    c->n_keys_used = 0;
    c->status &= ~(unsigned)(TTS_STATUS_KEY_OVERFLOW | TTS_STATUS_TIMEOUT);
    c->work_fwd = c->work_bwd = 0u;
    c->done_fwd = c->done_bwd = 0u;
    c->seg_total = 0;
    for (int q = 0; q < TSORT_CLASSES; ++q) c->class_n[q] = 0;
    for (int q = 0; q < 5; ++q) c->sort_q[q] = 0;
    c->scan_ticket = 0u;
  }
  const int nlb = (B->total_tiles + TS_TILES - 1) / TS_TILES;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nlb; t += gridDim.x * blockDim.x)
    B->scan_lb[t] = 0ull;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < B->total_tiles; t += gridDim.x * blockDim.x) {
    B->tile_cnt[t] = 0;
    if (B->tile_ovf) B->tile_ovf[t] = 0;
  }
}

// ---------------------------------------------------------------------------
// K1: pre-filter.  alpha_max = Eq. 1 at (f_max, f_min) of the tet's vertices,
// keep iff alpha_max >= T_f.  Flags, then a stable compaction.
// grid (max_pf_chunks, n_scenes).  A block first copies its chunk of tet
// indices into shared memory with asynchronous 16-byte copies (all in flight
// at once, evict-first in L2), then gathers the vertex SDF values.
// ---------------------------------------------------------------------------
// 16-byte asynchronous copy global -> shared that marks the L2 lines it
// brings in evict-first: the tet indices stream through once and should not
// push the vertex arrays (gathered right after) out of L2.
__device__ __forceinline__ void cp_async16_stream(void* smem, const void* gmem,
                                                  unsigned long long policy) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(sa),
               "l"(gmem), "l"(policy)
               : "memory");
}

__global__ void __launch_bounds__(PF_THREADS) k_prefilter_flags(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ int4 sT[PF_CHUNK];
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
  const int nk = (int)(k1 - k0);
  unsigned long long policy;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
  for (int i = threadIdx.x; i < nk; i += PF_THREADS) cp_async16_stream(&sT[i], &S.T[k0 + i], policy);
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  int cnt = 0;
  bool bad = false;
#pragma unroll 4
  for (int i = threadIdx.x; i < nk; i += PF_THREADS) {
    const long long k = k0 + i;
    const int4 t = sT[i];
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
  pdl_wait();
  pdl_launch_dependents();
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

// Stable compaction: survivors (tet ids and their vertex ids) in original
// tet order.
__global__ void __launch_bounds__(PF_THREADS) k_prefilter_compact(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int chunk = blockIdx.x;
  if (chunk >= S.pf_chunks) return;
  constexpr int PER = PF_CHUNK / PF_THREADS;  // 8 consecutive flags per thread
  static_assert(PER == 8, "one 8-byte load of flags per thread");
  const long long k0 = (long long)chunk * PF_CHUNK + (long long)threadIdx.x * PER;
  // flag_off and k0 are multiples of 8 and the flag region is padded to 16
  // bytes per scene, so a load that starts below K stays inside it; flags
  // past K are masked
  const uint2 w = (k0 < S.K) ? *reinterpret_cast<const uint2*>(B->pf_flags + S.flag_off + k0)
                             : make_uint2(0u, 0u);
  unsigned char fl[PER];
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const unsigned word = (q < 4) ? w.x : w.y;
    fl[q] = (k0 + q < S.K) ? (unsigned char)((word >> (8 * (q & 3))) & 0xffu) : 0;
    cnt += fl[q];
  }
  int total;
  int off = block_excl_scan<int, PF_THREADS>(cnt, &total) + B->pf_blocksum[S.pf_chunk_base + chunk];
  int* out = B->surv + S.surv_off;
  int4* outT = B->surv_T + S.surv_off;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (fl[q]) {
      if (off < S.surv_cap) {
        out[off] = (int)(k0 + q);
        outT[off] = __ldg(&S.T[k0 + q]);
      }
      ++off;
    }
  }
}

// Per-survivor world unit normal n = g / |g| of the tet's affine SDF (Sec. 3.2
// per-tet normal, App. A.3), view independent and hoisted into the scene
// preparation (App. B.1).  grid (blocks, n_scenes)
__global__ void __launch_bounds__(256) k_tet_normals(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int nsurv = B->ctr->n_surv[s];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nsurv; k += gridDim.x * blockDim.x) {
    const int4 t = B->surv_T[S.surv_off + k];
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
    const int4 t = B->surv_T[S.surv_off + k];
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
// Warp-aggregated bucket counter: every active lane adds one to bucket[gt];
// lanes with equal gt share one atomic.  Returns the lane's position among
// the bucket's additions (the old value plus its rank in its group).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_bucket_add(int* bucket, int gt, unsigned active, bool want_pos) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(active, gt);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) {
    if (want_pos) base = atomicAdd(bucket + gt, __popc(peers));
    else atomicAdd(bucket + gt, __popc(peers));
  }
  if (!want_pos) return 0;
  base = __shfl_sync(active, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------------------
// K2: preprocess.  grid (max_pre_chunks, n_scenes), one thread per survivor
// of a scene: the tet is loaded once, then for each of the scene's views the
// thread writes the slot's record, tile rect and depth bits, and counts the
// keys of every tile the slot's rect overlaps.
// ---------------------------------------------------------------------------
constexpr int PP_SMEM_VIEWS = 16;

template <bool HULL>
__global__ void __launch_bounds__(PRE_THREADS, 5) k_preprocess(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  const int sc = blockIdx.y;
  const SceneD& S = B->sc[sc];
  const int nsurv = B->ctr->n_surv[sc];
  const int k0 = blockIdx.x * PRE_CHUNK;
  if (k0 >= nsurv) return;
  __shared__ unsigned s_zmn, s_zmx;
  __shared__ int s_left;
  // each warp's 32 records of the current view, stored out coalesced
  __shared__ __align__(16) float4 s_rec[PRE_THREADS / 32][32 * REC_Q];
  // the scene's view constants in shared memory (up to PP_SMEM_VIEWS views)
  __shared__ ViewD s_vw[PP_SMEM_VIEWS];
  const int nv = S.view_cnt;
  const bool vs = nv <= PP_SMEM_VIEWS;
  if (threadIdx.x == 0) {
    s_zmn = 0xffffffffu;
    s_zmx = 0u;
    s_left = PRE_THREADS / 32;
  }
  if (vs) {
    constexpr int VW = sizeof(ViewD) / 4;
    for (int w = threadIdx.x; w < nv * VW; w += PRE_THREADS) {
      const int vi = w / VW;
      reinterpret_cast<int*>(s_vw)[w] =
          reinterpret_cast<const int*>(&B->vw[B->scene_views[S.view_off + vi]])[w - vi * VW];
    }
  }
  __syncthreads();
  const float s = B->s;
  const int tsh = __ffs(B->tile) - 1;   // tile is 8, 16 or 32
  unsigned zmn = 0xffffffffu, zmx = 0u;
  for (int q = threadIdx.x; q < PRE_CHUNK; q += PRE_THREADS) {
    const int k = k0 + q;
    if (!__any_sync(0xffffffffu, k < nsurv)) break;   // warps stay converged
    TetIn in;
    float3 colour = f3(0.f, 0.f, 0.f);
    if (k < nsurv) {
      load_tet_ids(S, B->surv_T[S.surv_off + k], in);
      colour = tet_colour(in.c);     // view independent: the vertex colours die here
    }
    // one view of the survivor: record, pixel rect, depth bits, tile counts
    auto view = [&](const ViewD& vw) {
      int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0, ntx = 0, nt = 0;
      unsigned mask = 0xffffffffu;
      if (k < nsurv) {
        const long long slot = vw.rec_base + k;
        Geo G;
        float pu[4], pv[4];
        G.visible = HULL ? key_path(vw, in, G, pu, pv) : key_path(vw, in, G);
        if (G.visible) tet_geometry_rest(vw, in, G);   // may find a flat tet (not visible)
        if (G.visible) {
          tx0 = G.i0 >> tsh;     // pixel bounds are >= 0
          ty0 = G.j0 >> tsh;
          tx1 = G.i1 >> tsh;
          ty1 = G.j1 >> tsh;
          ntx = tx1 - tx0 + 1;
          nt = ntx * (ty1 - ty0 + 1);
          write_record(vw, s, in, G, colour, &s_rec[threadIdx.x >> 5][(threadIdx.x & 31) * REC_Q]);
          // the hull test after the record (most of the geometry is dead by then)
          if constexpr (HULL) {
            mask = hull_tile_mask(pu, pv, G, tsh, tx0, ty0, ntx, ty1 - ty0 + 1);
            if (mask == 0u) nt = 0;   // no pixel centre of the bbox inside the hull
          }
          if (nt > 0) {
            zmn = min(zmn, G.zbits);
            zmx = max(zmx, G.zbits);
          }
        }
        // the rect of a culled slot is empty (x1 < x0): the placement reads
        // the rect (the hull's kept cells in the high halves of x and y) and
        // the depth bits only
        B->rec_rect[slot] = nt > 0 ? make_int4(tx0 | (int)((mask & 0xffffu) << 16),
                                               tx1 | (int)((mask >> 16) << 16), ty0, ty1)
                                   : make_int4(1, 0, 0, 0);
        B->rec_z[slot] = G.zbits;
      }
      // the warp's records: its slots are consecutive (k = k0 + 32 w + lane), the
      // lanes with k < nsurv a prefix; a record of an invisible slot is never read
      {
        __syncwarp();
        const int lane = threadIdx.x & 31;
        const int nvalid = __popc(__ballot_sync(0xffffffffu, k < nsurv));
        const long long slot0 = vw.rec_base + (k - lane);
        float4* __restrict__ dst = B->rec + slot0 * REC_Q;
        const float4* srcw = s_rec[threadIdx.x >> 5];
        for (int i = lane; i < nvalid * REC_Q; i += 32) dst[i] = srcw[i];
        __syncwarp();
      }
      // key counts per kept tile, one atomic per (warp, tile) and round
      int* __restrict__ cnt = B->tile_cnt + vw.tile_base;
      int cx = 0, cy = 0;    // position of round r in the rect
      const bool masked = nt <= 32;
      for (int r = 0; __any_sync(0xffffffffu, r < nt); ++r) {
        const bool kept = r < nt && (!masked || ((mask >> r) & 1u));
        const unsigned act = __ballot_sync(0xffffffffu, kept);
        if (kept) warp_bucket_add(cnt, (ty0 + cy) * vw.tiles_x + tx0 + cx, act, false);
        if (r < nt && ++cx == ntx) {
          cx = 0;
          ++cy;
        }
      }
    };
    if (vs) {
      for (int vi = 0; vi < nv; ++vi) view(s_vw[vi]);
    } else {
      for (int vi = 0; vi < nv; ++vi) view(B->vw[B->scene_views[S.view_off + vi]]);
    }
  }
  // block min/max of the depth bits without a block barrier: each warp adds
  // its own to shared memory, the block's last warp to do so adds the block's
  zmn = __reduce_min_sync(0xffffffffu, zmn);
  zmx = __reduce_max_sync(0xffffffffu, zmx);
  if ((threadIdx.x & 31) == 0) {
    if (zmn != 0xffffffffu) {
      atomicMin(&s_zmn, zmn);
      atomicMax(&s_zmx, zmx);
    }
    __threadfence_block();
    if (atomicAdd(&s_left, -1) == 1) {
      const unsigned mn = atomicOr(&s_zmn, 0u), mx = atomicOr(&s_zmx, 0u);
      if (mn != 0xffffffffu) {
        atomicMin(&B->ctr->zmin_bits, mn);
        atomicMax(&B->ctr->zmax_bits, mx);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K3: tile scan.  Exclusive prefix of the per-tile key counts -> each tile's
// [start, end) ((0, 0) when empty) and its placement cursor (= start); the
// tiles listed by list-length class; the total is the key count.  Blocks of
// TS_THREADS x TS_ITEMS tiles take tickets in order, publish their count
// sum, and find the sum of all earlier blocks by decoupled look-back (the
// waits are bounded: past B->ts_spin_limit polls the scan sets
// TTS_STATUS_TIMEOUT, and the kernels after it use no key, as on overflow).
// Past the key capacity the key count is set, the overflow status raised and
// no key is used (the work-list builder then empties every range).  The last
// block also fixes the depth bit count.
// ---------------------------------------------------------------------------
constexpr unsigned long long TS_AGG = 1ull << 62, TS_PREFIX = 2ull << 62;

// No key is used: the scan exceeded the key capacity or one of its waits gave
// up (both leave ranges and cursors that do not describe placed keys).
__device__ __forceinline__ bool keys_unusable(const Counters* c) {
  return c->n_keys_used == 0 || (c->status & TTS_STATUS_TIMEOUT) != 0u;
}

// List-length class of the per-tile depth sort (see K5): up to 256 keys,
// 512, 1,024, 2,048, 4,096, more.
__device__ __forceinline__ int tsort_class(int n) {
  return n <= 256 ? 0 : n <= 512 ? 1 : n <= 1024 ? 2 : n <= 2048 ? 3 : n <= 4096 ? 4 : 5;
}

__global__ void __launch_bounds__(TS_THREADS) k_tile_scan(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ int s_b;
  __shared__ long long s_excl;
  Counters* c = B->ctr;
  if (threadIdx.x == 0) s_b = (int)atomicAdd(&c->scan_ticket, 1u);
  __syncthreads();
  const int b = s_b;
  const int n = B->total_tiles;
  int* __restrict__ cnt = B->tile_cnt;
  int2* __restrict__ ranges = B->ranges;
  const int i0 = b * TS_TILES + threadIdx.x * TS_ITEMS;
  int v[TS_ITEMS];
  if (i0 + TS_ITEMS <= n) {
    const int4* p = reinterpret_cast<const int4*>(cnt + i0);
#pragma unroll
    for (int j = 0; j < TS_ITEMS / 4; ++j) {
      const int4 x = p[j];
      v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) v[j] = (i0 + j < n) ? cnt[i0 + j] : 0;
  }
  long long sum = 0;
#pragma unroll
  for (int j = 0; j < TS_ITEMS; ++j) sum += v[j];
  long long tot;
  const long long tex = block_excl_scan<long long, TS_THREADS>(sum, &tot);
  if (threadIdx.x == 0) {
    unsigned long long* lb = B->scan_lb;
    long long excl = 0;
    if (b > 0) {
      atomicExch(lb + b, TS_AGG | (unsigned long long)tot);
      bool timed_out = false;
      const long long limit = B->ts_spin_limit;
      for (int p = b - 1; p >= 0 && !timed_out;) {
        // the test hook: this block polls a word no block publishes
        const unsigned long long* src = (b == B->ts_unset_block) ? &c->scan_unset : lb + p;
        unsigned long long w = *reinterpret_cast<const volatile unsigned long long*>(src);
        long long spins = 0;
        while (w == 0ull) {
          if (++spins > limit) {
            timed_out = true;
            break;
          }
          w = *reinterpret_cast<const volatile unsigned long long*>(src);
        }
        if (timed_out) break;
        excl += (long long)(w & (TS_AGG - 1));
        if (w & TS_PREFIX) break;
        --p;
      }
      if (timed_out) set_status(c, TTS_STATUS_TIMEOUT);
    }
    atomicExch(lb + b, TS_PREFIX | (unsigned long long)(excl + tot));
    s_excl = excl;
  }
  __syncthreads();
  long long ex = s_excl + tex;
  int cls[TS_ITEMS];
#pragma unroll
  for (int j = 0; j < TS_ITEMS; ++j) {
    cls[j] = -1;
    if (i0 + j < n) {
      const bool keep = v[j] > 0 && ex + v[j] <= B->key_cap;
      ranges[i0 + j] = keep ? make_int2((int)ex, (int)(ex + v[j])) : make_int2(0, 0);
      cnt[i0 + j] = (int)min(ex, (long long)0x7fffffff);
      if (keep) cls[j] = tsort_class(v[j]);
    }
    ex += v[j];
  }
  // the non-empty tiles by list-length class (one atomic per warp and class)
#pragma unroll
  for (int q = 0; q < TSORT_CLASSES; ++q) {
    int nq = 0;
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) nq += (cls[j] == q);
    int wt;
    const int wx = warp_excl_scan(nq, &wt);
    int b0 = 0;
    if ((threadIdx.x & 31) == 0 && wt > 0) b0 = atomicAdd(&c->class_n[q], wt);
    int pos = __shfl_sync(0xffffffffu, b0, 0) + wx;
    int* list = B->tile_class + (size_t)q * n;
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j)
      if (cls[j] == q) list[pos++] = i0 + j;
  }
  if (threadIdx.x == 0 && b == gridDim.x - 1) {
    const long long total = s_excl + tot;
    const bool over = total > B->key_cap;
    c->n_keys = total;
    c->n_keys_used = over ? 0 : total;
    if (over) set_status(c, TTS_STATUS_KEY_OVERFLOW);
    unsigned span = (c->zmax_bits >= c->zmin_bits) ? (c->zmax_bits - c->zmin_bits) : 0u;
    if (c->zmin_bits == 0xffffffffu) span = 0;
    const int db = (span == 0) ? 0 : (32 - __clz(span));
    c->depth_bits = db;
    c->total_bits = db + B->tile_bits;
  }
}

// ---------------------------------------------------------------------------
// K4: key placement.  grid (max_pp_chunks, n_views).  Each (slot, overlapped
// tile) pair takes the next position of its tile's bucket (one atomic per
// warp and tile) and stores the composite (zbits << 32 | slot) there: the
// buckets hold the right keys, in an arbitrary order that the per-tile sort
// removes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PP_THREADS) k_place(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  const int v = blockIdx.y;
  const ViewD& vw = B->vw[v];
  const int chunk = blockIdx.x;
  if (chunk >= vw.pp_chunks) return;
  const Counters* c = B->ctr;
  const long long used = c->n_keys_used;
  if (keys_unusable(c)) return;
  const int nsurv = c->n_surv[vw.scene];
  int* __restrict__ cur = B->tile_cnt + vw.tile_base;
  unsigned long long* __restrict__ out = B->keys[1];
  for (int q = threadIdx.x; q < PP_CHUNK; q += PP_THREADS) {
    const int k = chunk * PP_CHUNK + q;
    if (!__any_sync(0xffffffffu, k < nsurv)) break;
    int nt = 0, ntx = 1;
    int4 r = make_int4(0, 0, 0, 0);
    unsigned mask = 0xffffffffu;
    unsigned long long comp = 0;
    if (k < nsurv) {
      const long long slot = vw.rec_base + k;
      r = B->rec_rect[slot];            // empty (x1 < x0) for a culled slot
      mask = ((unsigned)r.x >> 16) | ((unsigned)r.y & 0xffff0000u);   // kept cells (hull test)
      r.x &= 0xffff;
      r.y &= 0xffff;
      const unsigned zb = B->rec_z[slot];
      if (r.y >= r.x) {
        ntx = r.y - r.x + 1;
        nt = ntx * (r.w - r.z + 1);
        comp = ((unsigned long long)zb << 32) | (unsigned)slot;
      }
    }
    const bool masked = nt <= 32;
    int cx = 0, cy = 0;    // position of round j in the rect
    for (int j = 0; __any_sync(0xffffffffu, j < nt); ++j) {
      const bool kept = j < nt && (!masked || ((mask >> j) & 1u));
      const unsigned act = __ballot_sync(0xffffffffu, kept);
      if (kept) {
        const int pos = warp_bucket_add(cur, (r.z + cy) * vw.tiles_x + r.x + cx, act, true);
        if (pos < used) out[pos] = comp;
      }
      if (j < nt && ++cx == ntx) {
        cx = 0;
        ++cy;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K5: per-tile depth sort.  Within a tile the keys are ordered by the mean
// depth bits and, for equal depths, by slot (that is, survivor order): the
// order of a stable sort of the (tile, depth) keys in slot order.  Composite
// keys are distinct, so any correct sort gives that one order.
//
// A merge sort per list: each thread sorts K keys in registers, then runs of
// K, 2K, ... are merged pairwise through shared memory (each thread finds
// where its K outputs start on the merge path by binary search, then merges
// them sequentially).  Padding keys are all ones (no real key: the depth
// bits of a kept slot are those of a finite positive float).
//
// One persistent kernel of 256-thread blocks (four per SM) sorts every
// list, longest first: the tile scan lists the tiles by length class, and
// the blocks take (1) lists of more than 2,048 keys, one per block (more
// than 4,096: sorted runs of 4,096 merged in global memory), then lists of
// (2) 1,025..2,048 keys, one per half block, (3) 513..1,024, one per
// quarter block, (4) 257..512, one per warp, and (5) up to 256 keys, one per
// warp at 8 keys per lane, each from its own device queue.  A group sorts
// its list padded to 16 keys per thread (8 in (5)), so the finer classes
// bound the padding by the list length; 16 keys per thread take one merge
// round fewer and half the merge-path searches per key of 8.
// ---------------------------------------------------------------------------
constexpr int TSORT_NT = 256;

// Barrier of a group of NT threads: the warp, the whole block, or the named
// barrier bar of a half block (1, 2) or a quarter (3..6).
// Named barriers take immediate ids.
template <int NT>
__device__ __forceinline__ void group_sync(int bar) {
  if constexpr (NT == 32) {
    __syncwarp();
  } else if constexpr (NT == TSORT_NT) {
    __syncthreads();
  } else {
    switch (bar) {
#define TSORT_BAR(i) case i: asm volatile("bar.sync " #i ", %0;" ::"n"(NT) : "memory"); break;
      TSORT_BAR(1) TSORT_BAR(2) TSORT_BAR(3) TSORT_BAR(4) TSORT_BAR(5) TSORT_BAR(6)
#undef TSORT_BAR
      default: break;
    }
  }
}

// Shared-memory slot of key e: one pad key after every 16, so that the
// blocked accesses (thread t, key t K + q) of a half warp meet 16 distinct
// 8-byte bank pairs.
__device__ __forceinline__ int spad(int e) { return e + (e >> 4); }
template <int N>
__host__ __device__ constexpr int spad_size() { return N + N / 16; }

// Sorts the NT * K keys held K per thread (any arrangement) ascending; on
// return thread tid holds outputs [tid K, tid K + K).  s: spad_size(NT * K)
// keys of shared memory.
template <int NT, int K>
__device__ __forceinline__ void group_merge_sort(unsigned long long (&k)[K], unsigned long long* s,
                                                 int tid, int bar) {
  static_assert(K == 8 || K == 16, "the register networks sort 8 or 16 keys");
  // Batcher's odd-even merge network for 8 keys (19 compare-exchanges); for
  // 16, two of them and Batcher's merge of the two sorted halves (25 more)
  constexpr int NET[19][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6},
                              {5, 7}, {1, 2}, {5, 6}, {0, 4}, {1, 5}, {2, 6}, {3, 7},
                              {2, 4}, {3, 5}, {1, 2}, {3, 4}, {5, 6}};
  constexpr int MERGE16[25][2] = {{0, 8}, {4, 12}, {4, 8}, {2, 10}, {6, 14}, {6, 10}, {2, 4},
                                  {6, 8}, {10, 12}, {1, 9}, {5, 13}, {5, 9}, {3, 11}, {7, 15},
                                  {7, 11}, {3, 5}, {7, 9}, {11, 13}, {1, 2}, {3, 4}, {5, 6},
                                  {7, 8}, {9, 10}, {11, 12}, {13, 14}};
#pragma unroll
  for (int h = 0; h < K; h += 8) {
#pragma unroll
    for (int c = 0; c < 19; ++c) {
      const unsigned long long x = k[h + NET[c][0]], y = k[h + NET[c][1]];
      const bool sw = y < x;
      k[h + NET[c][0]] = sw ? y : x;
      k[h + NET[c][1]] = sw ? x : y;
    }
  }
  if constexpr (K == 16) {
#pragma unroll
    for (int c = 0; c < 25; ++c) {
      const unsigned long long x = k[MERGE16[c][0]], y = k[MERGE16[c][1]];
      const bool sw = y < x;
      k[MERGE16[c][0]] = sw ? y : x;
      k[MERGE16[c][1]] = sw ? x : y;
    }
  }
  for (int run = K; run < NT * K; run <<= 1) {
    // merges of runs within one warp's 32 K keys need only the warp's barrier
    const bool in_warp = 2 * run <= 32 * K;
#pragma unroll
    for (int i = 0; i < K; ++i) s[spad(tid * K + i)] = k[i];
    if (in_warp) __syncwarp();
    else group_sync<NT>(bar);
    const int d0 = tid * K;
    const int start = d0 & ~(2 * run - 1);
    const int d = d0 - start;
    const int a0 = start, b0 = start + run;
    int lo = max(0, d - run), hi = min(d, run);
    while (lo < hi) {                   // first i with b[d-1-i] < a[i]
      const int mid = (lo + hi) >> 1;
      if (!(s[spad(b0 + d - 1 - mid)] < s[spad(a0 + mid)])) lo = mid + 1;
      else hi = mid;
    }
    int i = lo, j = d - lo;
    unsigned long long va = (i < run) ? s[spad(a0 + i)] : ~0ull;
    unsigned long long vb = (j < run) ? s[spad(b0 + j)] : ~0ull;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      // branch free: one shared load per output, from the side that advanced
      const bool ta = (i < run) && (j >= run || !(vb < va));
      k[q] = ta ? va : vb;
      i += ta;
      j += !ta;
      const int nx = ta ? i : j;
      const int e = (ta ? a0 : b0) + nx;
      const unsigned long long nv = (nx < run) ? s[spad(e)] : ~0ull;
      va = ta ? nv : va;
      vb = ta ? vb : nv;
    }
    if (in_warp) __syncwarp();
    else group_sync<NT>(bar);
  }
}

// Loads in[0, n) (n <= NT * K, padded), sorts, and writes the slots of the
// sorted keys to out[0, n) (through shared memory, so the stores coalesce)
// or, when keys_out is given, the sorted keys there.
template <int NT, int K>
__device__ __forceinline__ void group_sort_list(const unsigned long long* in, int n, unsigned* out,
                                                unsigned long long* keys_out, unsigned long long* s,
                                                int tid, int bar) {
  unsigned long long k[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int i = q * NT + tid;
    k[q] = (i < n) ? in[i] : ~0ull;
  }
  group_merge_sort<NT, K>(k, s, tid, bar);
#pragma unroll
  for (int q = 0; q < K; ++q) s[spad(tid * K + q)] = k[q];
  group_sync<NT>(bar);
  for (int i = tid; i < n; i += NT) {
    if (keys_out) keys_out[i] = s[spad(i)];
    else out[i] = (unsigned)s[spad(i)];
  }
  group_sync<NT>(bar);
}

constexpr int TSORT_K = 16;
constexpr int TSORT_BLOCK_CAP = TSORT_NT * TSORT_K;        // 4,096
constexpr int TSORT_WARP_CAP = 32 * TSORT_K;               // 512
constexpr int TSORT_SMALL_K = 8;                           // lists of up to 256 keys

// Merge of the sorted runs a[0, la) and b[0, lb) into o[0, la + lb) by all
// threads of the block (merge path in global memory).
template <int NT>
__device__ void block_merge(const unsigned long long* a, int la, const unsigned long long* b, int lb,
                            unsigned long long* o) {
  const int total = la + lb;
  const int per = (total + NT - 1) / NT;
  const int d0 = threadIdx.x * per;
  if (d0 >= total) return;
  const int d1 = min(d0 + per, total);
  int lo = max(0, d0 - lb), hi = min(d0, la);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (!(b[d0 - 1 - mid] < a[mid])) lo = mid + 1;
    else hi = mid;
  }
  int i = lo, j = d0 - lo;
  for (int d = d0; d < d1; ++d) {
    const bool take_a = (i < la) && (j >= lb || !(b[j] < a[i]));
    o[d] = take_a ? a[i++] : b[j++];
  }
}

// A list of more than TSORT_BLOCK_CAP keys, by the whole block: sorted runs
// of TSORT_BLOCK_CAP keys, then block merges of run pairs between keys[1]
// and keys[0] (the block owns the tile's range in both).
__device__ void sort_long_list(const Batch* __restrict__ B, int2 r, unsigned long long* s) {
  const int n = r.y - r.x;
  unsigned long long* A = B->keys[1] + r.x;
  for (int c0 = 0; c0 < n; c0 += TSORT_BLOCK_CAP)
    group_sort_list<TSORT_NT, TSORT_K>(A + c0, min(TSORT_BLOCK_CAP, n - c0), nullptr, A + c0, s,
                                       threadIdx.x, 0);
  unsigned long long* src = A;
  unsigned long long* dst = B->keys[0] + r.x;
  for (int w = TSORT_BLOCK_CAP; w < n; w <<= 1) {
    for (int lo = 0; lo < n; lo += 2 * w) {
      const int mid = min(lo + w, n), hi = min(lo + 2 * w, n);
      block_merge<TSORT_NT>(src + lo, mid - lo, src + mid, hi - mid, dst + lo);
    }
    __syncthreads();
    unsigned long long* x = src;
    src = dst;
    dst = x;
  }
  for (int i = threadIdx.x; i < n; i += TSORT_NT) B->vals[r.x + i] = (unsigned)src[i];
  __syncthreads();
}

// Lists of one class, one per group of NT threads (group g of the block,
// named barrier bar), from device queue q; s: the group's shared memory.
template <int NT, int K = TSORT_K>
__device__ __forceinline__ void sort_group_lists(const Batch* __restrict__ B, int cls, int q,
                                                 int g, int bar, unsigned long long* s,
                                                 int* s_item) {
  Counters* c = B->ctr;
  const int n = c->class_n[cls];
  const int* list = B->tile_class + (size_t)cls * B->total_tiles;
  const unsigned long long* in = B->keys[1];
  const int tid = threadIdx.x & (NT - 1);
  for (;;) {
    if (tid == 0) s_item[g] = atomicAdd(&c->sort_q[q], 1);
    group_sync<NT>(bar);
    const int it = s_item[g];
    group_sync<NT>(bar);
    if (it >= n) break;
    const int2 r = B->ranges[list[it]];
    group_sort_list<NT, K>(in + r.x, r.y - r.x, B->vals + r.x, nullptr, s, tid, bar);
  }
}

__global__ void __launch_bounds__(TSORT_NT, TSORT_BLOCKS_PER_SM) k_tile_sort(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ unsigned long long s[spad_size<TSORT_BLOCK_CAP>()];
  __shared__ int s_item[16];
  Counters* c = B->ctr;
  if (keys_unusable(c)) return;
  const int nt = B->total_tiles;
  const int* list = B->tile_class;
  const int n5 = c->class_n[5], n4 = c->class_n[4], n0 = c->class_n[0];
  const unsigned long long* in = B->keys[1];
  // (1) lists of more than 2,048 keys (the longest class first), a block each
  for (;;) {
    if (threadIdx.x == 0) s_item[0] = atomicAdd(&c->sort_q[0], 1);
    __syncthreads();
    const int it = s_item[0];
    __syncthreads();
    if (it >= n5 + n4) break;
    const int t = (it < n5) ? list[5 * nt + it] : list[4 * nt + it - n5];
    const int2 r = B->ranges[t];
    if (r.y - r.x > TSORT_BLOCK_CAP) {
      if (threadIdx.x == 0) atomicAdd(&c->long_lists, 1);
      sort_long_list(B, r, s);
    } else {
      group_sort_list<TSORT_NT, TSORT_K>(in + r.x, r.y - r.x, B->vals + r.x, nullptr, s,
                                         threadIdx.x, 0);
    }
  }
  // (2) .. (4): halves, quarters, warps, each inside the shared memory of
  // the group it came from
  const int h = threadIdx.x >> 7, qd = threadIdx.x >> 6;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long* sw = s + w * spad_size<TSORT_WARP_CAP>();
  sort_group_lists<128>(B, 3, 1, h, 1 + h, s + h * spad_size<2048>(), s_item);
  sort_group_lists<64>(B, 2, 2, 2 + qd, 3 + qd, s + qd * spad_size<1024>(), s_item);
  sort_group_lists<32>(B, 1, 3, 6 + w, 0, sw, s_item);
  // (5) lists of up to 256 keys, a warp each (8 keys per lane), inside the
  // warp's share
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&c->sort_q[4], 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n0) break;
    const int2 r = B->ranges[list[it]];
    const int n = r.y - r.x;
    if (n == 1) {
      if (lane == 0) B->vals[r.x] = (unsigned)in[r.x];
      continue;
    }
    group_sort_list<32, TSORT_SMALL_K>(in + r.x, n, B->vals + r.x, nullptr, sw, lane, 0);
  }
}

// Debug view of the sorted lists as 64-bit keys (global tile << depth_bits |
// zbits - zmin_bits), rebuilt into keys[0] from the ranges and the slots'
// depth bits.  Not part of a render.
__global__ void k_debug_keys(const Batch* __restrict__ B) {
  const Counters* c = B->ctr;
  if (keys_unusable(c)) return;
  const int db = c->depth_bits;
  const unsigned zmin = c->zmin_bits;
  for (int t = blockIdx.x; t < B->total_tiles; t += gridDim.x) {
    const int2 r = B->ranges[t];
    for (int i = r.x + threadIdx.x; i < r.y; i += blockDim.x)
      B->keys[0][i] = ((unsigned long long)t << db) | (unsigned long long)(B->rec_z[B->vals[i]] - zmin);
  }
}

// Work lists for the persistent blend kernels.  A tile whose list is longer
// than seg_len entries is split into segments of seg_len entries: the forward
// walks the whole list as 4x2 blocks, in four units (tile, part << 24) of two
// blocks each (see fwd_lanes), and records its state at each segment end; the
// backward walks the segments in parallel from those states, one unit (tile,
// segment) each (one warp walking a long list back to front would otherwise
// bound its duration).  Another tile is one unit (tile, 0) of each list.
// Each list is ordered by decreasing work (bucketed by bit length: the
// forward's by list length, the backward's by list or segment length), so
// the longest start first; the order inside a bucket is arbitrary.

constexpr int WL_BUCKETS = 34;      // bit length of a work amount (0..32), 33: unused
constexpr int WL_COLS = 2 * WL_BUCKETS;   // forward buckets, then backward buckets
constexpr int WL_THREADS = 256;     // one tile per thread

__device__ __forceinline__ int wl_bucket(int n) { return n > 0 ? 32 - __clz(n) : 0; }

// Work-list step 1 (one tile per thread): segment count and checkpoint slots
// of each tile, and per block the units of each list and length bucket.
__global__ void __launch_bounds__(WL_THREADS) k_worklist_count(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ int cnt[WL_COLS];
  if (threadIdx.x < WL_COLS) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int t = blockIdx.x * WL_THREADS + threadIdx.x;
  const int nt = B->total_tiles;
  const int L = B->seg_len;
  const int lane = threadIdx.x & 31;
  const bool in = t < nt;
  // no key used (capacity exceeded): every list is empty
  const bool none = keys_unusable(B->ctr);
  int2 r = in ? B->ranges[t] : make_int2(0, 0);
  if (in && none && (r.x | r.y)) {
    r = make_int2(0, 0);
    B->ranges[t] = r;
  }
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
    B->tile_last[t] = 0;
    atomicAdd(&cnt[wl_bucket(len)], fwd_lanes(nseg));
    atomicAdd(&cnt[WL_BUCKETS + wl_bucket(nseg > 1 ? L : len)], nseg);
  }
  __syncthreads();
  if (threadIdx.x < WL_COLS) B->wl_blockcnt[blockIdx.x * WL_COLS + threadIdx.x] = cnt[threadIdx.x];
}

// Work-list step 2 (one block of 17 warps, four bucket columns each): per
// column, the exclusive prefix of the blocks' unit counts (in place) and, per
// list over its buckets from the longest down, the first unit of each bucket.
__global__ void __launch_bounds__(17 * 32) k_worklist_scan(const Batch* __restrict__ B, int nb) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ int total[WL_COLS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j < WL_COLS; j += 17) {
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
      const int b = b0 + lane;
      const int v = (b < nb) ? B->wl_blockcnt[b * WL_COLS + j] : 0;
      int tot;
      const int ex = warp_excl_scan(v, &tot);
      if (b < nb) B->wl_blockcnt[b * WL_COLS + j] = carry + ex;
      carry += tot;
    }
    if (lane == 0) total[j] = carry;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int l = threadIdx.x;
    int run = 0;
    for (int j = WL_BUCKETS - 1; j >= 0; --j) {
      B->wl_base[l * WL_BUCKETS + j] = run;
      run += total[l * WL_BUCKETS + j];
    }
    if (l == 0) B->ctr->n_units = run;
    else B->ctr->n_units_b = run;
  }
}

// Work-list step 3 (one tile per thread): each tile's units go after all
// units of longer buckets and after the earlier blocks' units of its bucket.
__global__ void __launch_bounds__(WL_THREADS) k_worklist_place(const Batch* __restrict__ B) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ int off[WL_COLS];
  if (threadIdx.x < WL_COLS)
    off[threadIdx.x] = B->wl_base[threadIdx.x] + B->wl_blockcnt[blockIdx.x * WL_COLS + threadIdx.x];
  __syncthreads();
  const int t = blockIdx.x * WL_THREADS + threadIdx.x;
  if (t >= B->total_tiles) return;
  const int L = B->seg_len;
  const int2 r = B->ranges[t];
  const int2 ts = B->tseg[t];
  const int len = r.y - r.x;
  const int parts = fwd_lanes(ts.y);         // forward units of the list
  const int pf = atomicAdd(&off[wl_bucket(len)], parts);
  for (int q = 0; q < parts; ++q) B->worklist[pf + q] = make_int2(t, q << 24);
  const int pb = atomicAdd(&off[WL_BUCKETS + wl_bucket(ts.y > 1 ? L : len)], ts.y);
  for (int j = 0; j < ts.y; ++j) B->worklist_b[pb + j] = make_int2(t, j);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_prefilter(const HostPlan& P, const Batch* dB, cudaStream_t st) {
  dim3 g(P.max_pf_chunks, P.n_scenes);
  launch_k(k_prefilter_flags, dim3(g), dim3(PF_THREADS), 0, st, dB);
  launch_k(k_prefilter_scan, dim3(1), dim3(SCAN_THREADS), 0, st, dB);
  launch_k(k_prefilter_compact, dim3(g), dim3(PF_THREADS), 0, st, dB);
  if (P.normals) {
    launch_k(k_tet_normals, dim3(P.normal_blocks, P.n_scenes), dim3(256), 0, st, dB);
    return 4;
  }
  return 3;
}

int launch_binning(const HostPlan& P, const Batch* dB, cudaStream_t st) {
  launch_k(k_fwd_reset, dim3(64), dim3(256), 0, st, dB);
  dim3 g(P.max_pp_chunks, P.n_views);
  if (P.hull)
    launch_k(k_preprocess<true>, dim3(P.max_pre_chunks, P.n_scenes), dim3(PRE_THREADS), 0, st, dB);
  else
    launch_k(k_preprocess<false>, dim3(P.max_pre_chunks, P.n_scenes), dim3(PRE_THREADS), 0, st, dB);
  launch_k(k_tile_scan, dim3((P.total_tiles + TS_TILES - 1) / TS_TILES), dim3(TS_THREADS), 0, st, dB);
  launch_k(k_place, dim3(g), dim3(PP_THREADS), 0, st, dB);
  launch_k(k_tile_sort, dim3(P.tsort_blocks), dim3(TSORT_NT), 0, st, dB);
  launch_k(k_worklist_count, dim3(P.wl_blocks), dim3(WL_THREADS), 0, st, dB);
  launch_k(k_worklist_scan, dim3(1), dim3(17 * 32), 0, st, dB, P.wl_blocks);
  launch_k(k_worklist_place, dim3(P.wl_blocks), dim3(WL_THREADS), 0, st, dB);
  return 8;
}

int launch_debug_keys(const HostPlan& P, const Batch* dB, cudaStream_t st) {
  k_debug_keys<<<P.tsort_blocks, 256, 0, st>>>(dB);
  return 1;
}

}  // namespace tts
