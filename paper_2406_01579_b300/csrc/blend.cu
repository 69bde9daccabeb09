// Per-tile blending (Eq. 1 opacity of each pixel's chord, Eq. 2 compositing
// with the 3DGS conventions), its backward, and the record -> vertex adjoint.
#include "geometry.cuh"
#include "launch.h"

namespace tts {

constexpr int WPB = 4;              // warps per block of the resort-window blend kernels and the
                                    // default of the others (tts_params.blend_warps: 2, 4 or 8)
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int find_view(const Batch* __restrict__ B, int gt) {
  int lo = 0, hi = B->n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B->vw[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Next work item for this warp from a global queue.
__device__ __forceinline__ int next_item(unsigned* counter) {
  int it = 0;
  if ((threadIdx.x & 31) == 0) it = (int)atomicAdd(counter, 1u);
  return __shfl_sync(FULL, it, 0);
}

// The last warp to leave resets the queue (and the optional second queue
// `extra`) so the next launch starts at 0.
__device__ __forceinline__ void queue_done(unsigned* counter, unsigned* done,
                                           unsigned* extra = nullptr) {
  if ((threadIdx.x & 31) == 0) {
    __threadfence();
    const unsigned total = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(done, 1u) == total - 1u) {
      *counter = 0u;
      if (extra) *extra = 0u;
      *done = 0u;
      __threadfence();
    }
  }
}

// The vertex-gradient arrays of a following record -> vertex scatter, cleared
// by the backward's warps once its work queue is empty (chunks of ZCH floats
// from the device queue q), so the clearing overlaps the longest walks.
// zg.dV[0] == nullptr: nothing to clear.
constexpr int ZCH = 4096;

__device__ __forceinline__ void zero_tail(const Batch* __restrict__ B, const GradOut& zg,
                                          unsigned* q) {
  if (zg.dV[0] == nullptr) return;
  const int lane = threadIdx.x & 31;
  for (;;) {
    long long ch = next_item(q);
    float* p = nullptr;
    long long len = 0;
    for (int s = 0; s < B->n_scenes && !p; ++s) {
      const long long N = B->sc[s].N;
      float* const arr[3] = {zg.dV[s], zg.df[s], zg.drgb[s]};
      const long long n[3] = {3 * N, N, 3 * N};
      for (int a = 0; a < 3; ++a) {
        const long long nch = (n[a] + ZCH - 1) / ZCH;
        if (ch < nch) {
          p = arr[a];
          len = n[a];
          break;
        }
        ch -= nch;
      }
    }
    if (!p) break;
    const long long i1 = min((ch + 1) * ZCH, len);
    for (long long i = ch * ZCH + lane; i < i1; i += 32) p[i] = 0.f;
  }
}

// A warp's work item: one 8x4 pixel block of one tile, lanes row-major.
struct WarpBlock {
  int gt;
  int seg;                    // segment of a split tile list (0 otherwise)
  int sb;                     // 8x4 block within the tile
  int part;                   // forward part of a long list (4x2 blocks part*SB ..)
  int tpix;                   // the lane's pixel within the tile, row-major
  int px, py;
  bool inimg;
  float fpx, fpy;
  float wx0, wx1, wy0, wy1;   // the block's pixel-centre rectangle
  unsigned lmask;             // the lanes the rectangle was taken over
  __device__ __forceinline__ bool misses(const float4& q0) const {
    return (fabsf(q0.x) > wx1) | (q0.z < wx0) | (fabsf(q0.y) > wy1) | (q0.w < wy0);
  }
  // Shrink the test rectangle to the pixels of the lanes in `live`: an entry
  // whose bbox misses all of them cannot produce a fragment for any lane that
  // still needs one.  Returns false when no lane is live.  The rectangle is
  // taken again only when the set of live lanes has changed.
  __device__ __forceinline__ bool cull_to(bool live) {
    const unsigned lm = __ballot_sync(FULL, live);
    if (lm == lmask) return lm != 0u;
    lmask = lm;
    if (lm == 0u) return false;
    const unsigned big = 0x7fffffffu;
    const unsigned x0 = __reduce_min_sync(FULL, live ? (unsigned)px : big);
    const unsigned x1 = __reduce_max_sync(FULL, live ? (unsigned)px : 0u);
    const unsigned y0 = __reduce_min_sync(FULL, live ? (unsigned)py : big);
    const unsigned y1 = __reduce_max_sync(FULL, live ? (unsigned)py : 0u);
    wx0 = (float)x0 + 0.5f;
    wx1 = (float)x1 + 0.5f;
    wy0 = (float)y0 + 0.5f;
    wy1 = (float)y1 + 0.5f;
    return true;
  }
};

// The warp block (tile gt, 8x4 block sb, list segment seg), lanes row-major.
template <int TILE>
__device__ __forceinline__ const ViewD& decode_block(const Batch* __restrict__ B, int gt, int seg,
                                                     int sb, WarpBlock& wb) {
  constexpr int SBX = TILE / 8;
  wb.gt = gt;
  wb.seg = seg;
  wb.sb = sb;
  wb.part = 0;
  const ViewD& vw = B->vw[find_view(B, wb.gt)];
  const int lt = wb.gt - vw.tile_base;
  const int tyi = lt / vw.tiles_x, txi = lt - tyi * vw.tiles_x;
  const int ox = (sb % SBX) * 8, oy = (sb / SBX) * 4;
  const int lane = threadIdx.x & 31;
  wb.tpix = (oy + (lane >> 3)) * TILE + ox + (lane & 7);
  const int bx = txi * TILE + ox, by = tyi * TILE + oy;
  wb.px = bx + (lane & 7);
  wb.py = by + (lane >> 3);
  wb.inimg = (wb.px < vw.W) & (wb.py < vw.H);
  wb.fpx = (float)wb.px + 0.5f;
  wb.fpy = (float)wb.py + 0.5f;
  wb.lmask = FULL;             // the whole block
  wb.wx0 = (float)bx + 0.5f;
  wb.wx1 = wb.wx0 + 7.f;
  wb.wy0 = (float)by + 0.5f;
  wb.wy1 = wb.wy0 + 3.f;
  return vw;
}

// A 4x2 pixel block (b8 in tile-local row-major order of 4x2 blocks) with
// four lanes per pixel: lane = 4 * (4 * row + column) + sub.
template <int TILE>
__device__ __forceinline__ const ViewD& decode_block8(const Batch* __restrict__ B, int gt, int b8,
                                                      WarpBlock& wb) {
  constexpr int BX = TILE / 4;
  wb.gt = gt;
  wb.seg = 0;
  wb.sb = 0;
  wb.part = 1;
  const ViewD& vw = B->vw[find_view(B, wb.gt)];
  const int lt = wb.gt - vw.tile_base;
  const int tyi = lt / vw.tiles_x, txi = lt - tyi * vw.tiles_x;
  const int ox = (b8 % BX) * 4, oy = (b8 / BX) * 2;
  const int pix = (threadIdx.x & 31) >> 2;
  wb.tpix = (oy + (pix >> 2)) * TILE + ox + (pix & 3);
  const int bx = txi * TILE + ox, by = tyi * TILE + oy;
  wb.px = bx + (pix & 3);
  wb.py = by + (pix >> 2);
  wb.inimg = (wb.px < vw.W) & (wb.py < vw.H);
  wb.fpx = (float)wb.px + 0.5f;
  wb.fpy = (float)wb.py + 0.5f;
  wb.lmask = FULL;             // the whole block
  wb.wx0 = (float)bx + 0.5f;
  wb.wx1 = wb.wx0 + 3.f;
  wb.wy0 = (float)by + 0.5f;
  wb.wy1 = wb.wy0 + 1.f;
  return vw;
}

// Work item -> warp block: item / SB indexes a work list of units (tile,
// segment | part << 24): the forward's (tile, part << 24), the parts of a long
// list covering its 4x2 blocks, or the backward's (tile, segment).
template <int TILE>
__device__ __forceinline__ const ViewD& decode_item(const Batch* __restrict__ B,
                                                    const int2* __restrict__ list, int item,
                                                    WarpBlock& wb) {
  constexpr int SB = (TILE / 8) * (TILE / 4);
  const int2 u = list[item / SB];
  const ViewD& vw = decode_block<TILE>(B, u.x, u.y & 0xffffff, item - (item / SB) * SB, wb);
  wb.part = u.y >> 24;
  return vw;
}

// Record-field gradients of one fragment, added into its slot's six float4
// (face major): row q < 4 holds face q's plane terms (dP, dA, dB) and, for
// q < 3, component q of the normal gradient in .w; row 4 the opacity terms
// (dF, dK0, dKx, dKy); row 5 depth and colour.  Only the chord's entry and
// exit faces (kin in 0..2, kout in 1..3, never equal) have nonzero plane
// terms, so a fragment takes four vector atomics; with normals, the
// components that neither face row carried go as scalar atomics.
template <bool NRM>
__device__ __forceinline__ void add_frag_grad(float4* __restrict__ dst, int kin, int kout,
                                              float dpin, float dpout, float cdx, float cdy,
                                              float4 r4, float4 r5, float gn0, float gn1,
                                              float gn2) {
  const float win = NRM ? (kin == 0 ? gn0 : (kin == 1 ? gn1 : gn2)) : 0.f;
  const float wout = NRM ? (kout == 1 ? gn1 : (kout == 2 ? gn2 : 0.f)) : 0.f;
  atomicAdd(dst + kin, make_float4(dpin, dpin * cdx, dpin * cdy, win));
  atomicAdd(dst + kout, make_float4(dpout, dpout * cdx, dpout * cdy, wout));
  atomicAdd(dst + 4, r4);
  atomicAdd(dst + 5, r5);
  if constexpr (NRM) {
    if (kin != 0) atomicAdd(&dst[0].w, gn0);
    if (kin != 1 && kout != 1) atomicAdd(&dst[1].w, gn1);
    if (kin != 2 && kout != 2) atomicAdd(&dst[2].w, gn2);
  }
}

// Per-slot normals of a view's tile lists: the survivor normals of its scene
// (slot - rec_base is the survivor index).
template <bool NRM>
__device__ __forceinline__ const float4* surv_normals(const Batch* __restrict__ B,
                                                      const ViewD& vw) {
  if constexpr (NRM) return B->surv_n + (B->sc[vw.scene].surv_off - vw.rec_base);
  return nullptr;
}

// Normal map output (planar like the image) and, when a backward follows,
// the final per-pixel normal.
__device__ __forceinline__ void store_normal(const Batch* __restrict__ B, const ViewD& vw,
                                             long long p, float* __restrict__ normal, float N0,
                                             float N1, float N2) {
  const long long HW = (long long)vw.W * vw.H;
  normal[3 * vw.pix_base + p] = N0;
  normal[3 * vw.pix_base + HW + p] = N1;
  normal[3 * vw.pix_base + 2 * HW + p] = N2;
  if (B->pix_N) B->pix_N[vw.pix_base + p] = make_float4(N0, N1, N2, 0.f);
}

// Per-pixel compositing state of the forward.  fl: the pixel's fragment list
// (record slots of its blended fragments, at most frag_cap of them; null when
// the batch keeps no lists), nb: its blended fragments so far.
struct FwdState {
  float T, C0, C1, C2, D, N0, N1, N2;
  int last, nfrag;
  bool done;
  int nb;
  unsigned* fl;
};

// Final per-pixel outputs of the forward.
template <bool NRM>
__device__ __forceinline__ void store_pixel(const Batch* __restrict__ B, const ViewD& vw,
                                            const WarpBlock& wb, const FwdState& S,
                                            float* __restrict__ image, float* __restrict__ alpha,
                                            float* __restrict__ depth, float* __restrict__ normal) {
  const long long HW = (long long)vw.W * vw.H;
  const long long p = (long long)wb.py * vw.W + wb.px;
  image[3 * vw.pix_base + p] = S.C0;
  image[3 * vw.pix_base + HW + p] = S.C1;
  image[3 * vw.pix_base + 2 * HW + p] = S.C2;
  alpha[vw.pix_base + p] = 1.f - S.T;
  depth[vw.pix_base + p] = S.D;
  B->pix_T[vw.pix_base + p] = S.T;
  B->pix_last[vw.pix_base + p] = S.last;
  B->pix_nfrag[vw.pix_base + p] = S.nfrag;
  B->pix_CD[vw.pix_base + p] = make_float4(S.C0, S.C1, S.C2, S.D);
  if (B->pix_nb) {
    B->pix_nb[vw.pix_base + p] = S.nb;
    if (S.nb > B->frag_cap) {   // the backward re-walks this tile's list
      B->tile_ovf[wb.gt] = 1;
      B->ctr->ovf_any = 1u;
    }
  }
  if constexpr (NRM) store_normal(B, vw, p, normal, S.N0, S.N1, S.N2);
}

// Fragment codes handed between the lanes of a pixel: alpha' > 0 (blend),
// FRAG_ZERO (blend with alpha' = 0), FRAG_SKIP (a chord, not blended), 0 (no
// chord).
constexpr float FRAG_ZERO = -2.f;
constexpr float FRAG_SKIP = -1.f;

// One fragment of the pixel's compositing (Eq. 2, 3DGS conventions), given
// its code v: counts the chord, blends alpha' or stops the pixel.
template <bool NRM>
__device__ __forceinline__ void composite(float v, int k, int base, bool pure, float eps,
                                          float4 (*st)[32], const int* sidx,
                                          const unsigned* sslot, int fcap, FwdState& S) {
  if (v == 0.f || S.done) return;
  ++S.nfrag;
  if (v == FRAG_SKIP) return;
  const float a = fmaxf(v, 0.f);
  const float Tn = __fmul_rn(S.T, __fsub_rn(1.f, a));
  if (!pure && Tn < eps) {
    S.done = true;
    return;
  }
  const float4 q5 = st[5][k];
  const float wgt = __fmul_rn(S.T, a);
  S.C0 = __fmaf_rn(wgt, q5.y, S.C0);
  S.C1 = __fmaf_rn(wgt, q5.z, S.C1);
  S.C2 = __fmaf_rn(wgt, q5.w, S.C2);
  S.D = __fmaf_rn(wgt, q5.x, S.D);
  if constexpr (NRM) {
    const float4 n = st[REC_Q][k];
    S.N0 = __fmaf_rn(wgt, n.x, S.N0);
    S.N1 = __fmaf_rn(wgt, n.y, S.N1);
    S.N2 = __fmaf_rn(wgt, n.z, S.N2);
  }
  S.T = Tn;
  S.last = base + sidx[k] + 1;
  if (fcap > 0) {   // (a done pixel, or one outside the image, never gets here)
    if (S.nb < fcap) S.fl[S.nb] = sslot[k];
    ++S.nb;
  }
}

// Eq. 1 with the cap and skip decisions, as a fragment code.
__device__ __forceinline__ float fragment_code(const float4& q4, const Chord& ch, bool pure,
                                               float cap, float skip) {
  const Opacity o = opacity_eval(q4, ch);
  const float a = pure ? o.alpha : fminf(o.alpha, cap);
  const bool use = pure ? (a > 0.f) : (a >= skip);
  return use ? (a > 0.f ? a : FRAG_ZERO) : FRAG_SKIP;
}

// LPP = 4: the four lanes of a pixel hold the fragment codes v of four
// consecutive candidates (lane sub has the sub-th).  The pixel's compositing
// of the four in order (as composite() one after the other): the
// transmittance in front of each is T times a product over the lanes before
// it (a scan over the four lanes), the first lane whose fragment would take
// T below eps stops the pixel, and each lane before it adds its own
// fragment to its partial colour / depth / normal sums (a pixel's sums are
// those of its four lanes).  T, done agree over the four lanes.
template <bool NRM>
__device__ __forceinline__ void composite4(float v, int k, int base, bool pure, float eps,
                                           float4 (*st)[32], const int* sidx,
                                           const unsigned* sslot, int fcap, FwdState& S) {
  const int lane = threadIdx.x & 31, sub = lane & 3, g0 = lane & ~3;
  const bool bl = (v != 0.f) & (v != FRAG_SKIP);
  const float a = bl ? fmaxf(v, 0.f) : 0.f;
  float P = bl ? __fsub_rn(1.f, a) : 1.f;        // inclusive product of (1 - a)
  float t = __shfl_up_sync(FULL, P, 1, 4);
  if (sub >= 1) P = __fmul_rn(t, P);
  t = __shfl_up_sync(FULL, P, 2, 4);
  if (sub >= 2) P = __fmul_rn(t, P);
  float Pex = __shfl_up_sync(FULL, P, 1, 4);      // exclusive
  if (sub == 0) Pex = 1.f;
  const float Tn = __fmul_rn(S.T, P);
  const bool stop = bl && !pure && (Tn < eps);
  const unsigned sbits = (__ballot_sync(FULL, stop) >> g0) & 0xfu;
  const int f = sbits ? __ffs(sbits) - 1 : 4;     // the first stopping lane (4: none)
  const float Tl = __shfl_sync(FULL, Tn, g0 + max(f - 1, 0));
  // the pixel's blended fragments of this group, in list (lane) order
  if (fcap > 0) {   // the same for the whole batch; a done pixel never blends
    const bool blend = bl && sub < f && !S.done;
    const unsigned bm = (__ballot_sync(FULL, blend) >> g0) & 0xfu;
    const int at = S.nb + __popc(bm & ((1u << sub) - 1u));
    if (blend && at < fcap) S.fl[at] = sslot[k];
    S.nb += __popc(bm);
  }
  if (S.done) return;
  S.nfrag += (v != 0.f) && sub <= f;
  if (bl && sub < f) {
    const float4 q5 = st[5][k];
    const float wgt = __fmul_rn(__fmul_rn(S.T, Pex), a);
    S.C0 = __fmaf_rn(wgt, q5.y, S.C0);
    S.C1 = __fmaf_rn(wgt, q5.z, S.C1);
    S.C2 = __fmaf_rn(wgt, q5.w, S.C2);
    S.D = __fmaf_rn(wgt, q5.x, S.D);
    if constexpr (NRM) {
      const float4 n = st[REC_Q][k];
      S.N0 = __fmaf_rn(wgt, n.x, S.N0);
      S.N1 = __fmaf_rn(wgt, n.y, S.N1);
      S.N2 = __fmaf_rn(wgt, n.z, S.N2);
    }
    S.last = base + sidx[k] + 1;
  }
  if (f >= 1) S.T = Tl;
  S.done = f < 4;
}

// Sum (max) of a value over the LPP lanes of a pixel.
template <int LPP>
__device__ __forceinline__ float pix_sum(float x) {
  if constexpr (LPP == 4) {
    x += __shfl_xor_sync(FULL, x, 1);
    x += __shfl_xor_sync(FULL, x, 2);
  }
  return x;
}
template <int LPP>
__device__ __forceinline__ int pix_sum_i(int x) {
  if constexpr (LPP == 4) {
    x += __shfl_xor_sync(FULL, x, 1);
    x += __shfl_xor_sync(FULL, x, 2);
  }
  return x;
}
template <int LPP>
__device__ __forceinline__ int pix_max_i(int x) {
  if constexpr (LPP == 4) {
    x = max(x, __shfl_xor_sync(FULL, x, 1));
    x = max(x, __shfl_xor_sync(FULL, x, 2));
  }
  return x;
}

// Walks the list entries [lo, hi) of the warp's tile front to back for the
// lanes that are not done: the entries whose bbox meets a live pixel are
// staged (ballot) in the warp's shared-memory slice and blended in order
// (Eq. 1 opacity, Eq. 2 compositing, 3DGS conventions); a pixel stops before
// the fragment that would take T below eps (not in PURE mode).  LPP = 1 (an
// 8x4 block, one lane per pixel): candidates in pairs; each lane evaluates
// both chords, then (when either meets a live lane) both opacities, then
// composites the two in order.  LPP = 4 (a 4x2 block, four lanes per pixel):
// candidates in fours; each lane of a pixel evaluates one of them, the four
// exchange their fragment codes and all composite the four in order, which
// cuts the chain a long list puts on one warp by four.  `last`
// counts list entries from lo.  When the list is split into segments for
// the backward (ts.y > 1), the state at the end of each segment is stored as
// the walk passes it.
template <bool NRM, int LPP, bool CNT>
__device__ __forceinline__ void fwd_walk(const Batch* __restrict__ B, WarpBlock wb,
                                         const unsigned* __restrict__ vals,
                                         const float4* __restrict__ rec,
                                         const float4* __restrict__ nrm, int lo, int hi, int2 ts,
                                         int tt, bool pure, float cap, float skip, float eps,
                                         float4 (*st)[32], int* sidx, unsigned* sslot, int fcap,
                                         FwdState& S) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LPP - 1);
  const unsigned ltm = (1u << lane) - 1u;
  const int L = B->seg_len;
  const bool split = ts.y > 1;
  // TTS_FLAG_COUNT (diagnostics, an instantiation of its own): one atomic per group
  constexpr bool count = CNT;
  if (count && lane == 0) atomicAdd(B->ctr->walk + 2, 1ull);
  // one group of lookahead on (slot, bbox)
  int idx = lo + lane;
  unsigned slot = (idx < hi) ? vals[idx] : 0u;
  float4 q0 = (idx < hi) ? __ldg(rec + (size_t)slot * REC_Q) : make_float4(0.f, 0.f, -1.f, -1.f);
  unsigned slot_n = (idx + 32 < hi) ? vals[idx + 32] : 0u;
  int gck = split ? lo + L : hi;   // the next segment end (L is a multiple of 32)
  long long pck = (long long)ts.x * tt + wb.tpix;
  for (int g = lo; g < hi; g += 32) {
    if (g == gck) {
      const float c0 = pix_sum<LPP>(S.C0), c1 = pix_sum<LPP>(S.C1), c2 = pix_sum<LPP>(S.C2);
      const float d = pix_sum<LPP>(S.D);
      float n0 = 0.f, n1 = 0.f, n2 = 0.f;
      if constexpr (NRM) {
        n0 = pix_sum<LPP>(S.N0);
        n1 = pix_sum<LPP>(S.N1);
        n2 = pix_sum<LPP>(S.N2);
      }
      if (sub == 0) {
        B->pseg_a[pck] = make_float4(S.T, c0, c1, c2);
        B->pseg_b[pck] = make_float4(d, n0, n1, n2);
      }
      gck += L;
      pck += tt;
    }
    if (!wb.cull_to(!S.done)) break;
    const int idn = g + 32 + lane;
    const float4 q0_n = (idn < hi) ? __ldg(rec + (size_t)slot_n * REC_Q)
                                   : make_float4(0.f, 0.f, -1.f, -1.f);
    const unsigned slot_nn = (idn + 32 < hi) ? vals[idn + 32] : 0u;
    const bool ov = (g + lane < hi) && !wb.misses(q0);
    const unsigned m = __ballot_sync(FULL, ov);
    if (count && lane == 0) {
      atomicAdd(B->ctr->walk + 0, 1ull);
      atomicAdd(B->ctr->walk + 1, (unsigned long long)__popc(m));
    }
    if (m != 0u) {
      if (ov) {
        const int pos = __popc(m & ltm);
        const float4* r = rec + (size_t)slot * REC_Q;
        st[0][pos] = q0;
#pragma unroll
        for (int q = 1; q < REC_Q; ++q) st[q][pos] = __ldg(r + q);
        if constexpr (NRM) st[REC_Q][pos] = __ldg(nrm + slot);
        sidx[pos] = lane;
        sslot[pos] = slot;
      }
      __syncwarp();
      const int cnt = __popc(m);
      const int base = g - lo;
      constexpr int STEP = (LPP == 4) ? 4 : 2;
      for (int k0 = 0; k0 < cnt; k0 += STEP) {
        if constexpr (LPP == 1) {
          const int ka = k0, kb = min(k0 + 1, cnt - 1);   // past the end: evaluated again, masked
          const Chord cha = chord_eval(st[0][ka], st[1][ka], st[2][ka], st[3][ka], wb.fpx, wb.fpy);
          const Chord chb = chord_eval(st[0][kb], st[1][kb], st[2][kb], st[3][kb], wb.fpx, wb.fpy);
          const bool ha = cha.hit, hb = chb.hit && (k0 + 1 < cnt);
          if (!__any_sync(FULL, (ha || hb) && !S.done)) continue;
          const float va = fragment_code(st[4][ka], cha, pure, cap, skip);
          const float vb = fragment_code(st[4][kb], chb, pure, cap, skip);
          composite<NRM>(ha ? va : 0.f, ka, base, pure, eps, st, sidx, sslot, fcap, S);
          composite<NRM>(hb ? vb : 0.f, kb, base, pure, eps, st, sidx, sslot, fcap, S);
        } else {
          const int k = min(k0 + sub, cnt - 1);
          const Chord ch = chord_eval(st[0][k], st[1][k], st[2][k], st[3][k], wb.fpx, wb.fpy);
          const bool h = ch.hit && (k0 + sub < cnt);
          // every lane evaluates its candidate's code (no divergence before the
          // pixel's exchange); a miss codes 0
          const float code = fragment_code(st[4][k], ch, pure, cap, skip);
          const float mine = h ? code : 0.f;
          // no lane blends: only the chord counts change
          if (!__any_sync(FULL, (mine != 0.f) & (mine != FRAG_SKIP))) {
            if (!S.done) S.nfrag += (mine != 0.f);
            continue;
          }
          composite4<NRM>(mine, k, base, pure, eps, st, sidx, sslot, fcap, S);
        }
        // with four lanes per pixel a group is short: the walk checks for an
        // all-stopped block once per group of 32 entries only
        if (LPP == 1 && __all_sync(FULL, S.done)) break;
      }
      __syncwarp();
    }
    slot = slot_n;
    q0 = q0_n;
    slot_n = slot_nn;
  }
}

// The backward's task list: every pixel of the warp block (lanes with `own`)
// whose fragment list holds all of its 1..fcap blended fragments, one
// atomic per warp.
__device__ __forceinline__ void list_pixel(const Batch* __restrict__ B, const ViewD& vw,
                                           const WarpBlock& wb, int nb, int fcap, bool own) {
  const bool want = own && wb.inimg && nb > 0 && nb <= fcap;
  const unsigned m = __ballot_sync(FULL, want);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  unsigned base = 0u;
  if (lane == leader) base = atomicAdd(&B->ctr->px_n, (unsigned)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (want)
    B->px_list[base + __popc(m & ((1u << lane) - 1u))] =
        make_uint2((unsigned)(vw.pix_base + (long long)wb.py * vw.W + wb.px),
                   (unsigned)nb | ((unsigned)(&vw - B->vw) << 8));
}

// ---------------------------------------------------------------------------
// K6: forward blend.  Persistent warps take work items from a queue (longest
// lists first), each one 8x4 pixel block of one tile list, and walk the list
// front to back (fwd_walk).  Units of the backward's later list segments
// (segment index > 0) have no forward work.
// ---------------------------------------------------------------------------
template <int TILE, bool NRM, int NW, bool CNT = false>
__global__ void __launch_bounds__(NW * 32) k_blend_fwd(const Batch* __restrict__ B,
                                                      float* __restrict__ image,
                                                      float* __restrict__ alpha,
                                                      float* __restrict__ depth,
                                                      float* __restrict__ normal) {
  pdl_wait();
  pdl_launch_dependents();
  constexpr int SB = (TILE / 8) * (TILE / 4);
  __shared__ float4 st[NW][REC_Q + NRM][32];
  __shared__ int sidx[NW][32];
  __shared__ unsigned sslot[NW][32];
  const int wid = threadIdx.x >> 5;
  Counters* c = B->ctr;
  const unsigned* __restrict__ vals = B->vals;
  const float4* __restrict__ rec = B->rec;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap, skip = B->alpha_skip, eps = B->t_eps;
  const int fcap = B->frag_cap;
  const int total = c->n_units * SB;
  for (int item = next_item(&c->work_fwd); item < total; item = next_item(&c->work_fwd)) {
    WarpBlock wb;
    const ViewD* vwp = &decode_item<TILE>(B, B->worklist, item, wb);
    const int2 ts = B->tseg[wb.gt];
    const int2 rg = B->ranges[wb.gt];
    // a long list: 4x2 blocks with four lanes per pixel (four forward units)
    const bool four = fwd_lanes(ts.y) == 4;
    if (four) vwp = &decode_block8<TILE>(B, wb.gt, wb.part * SB + wb.sb, wb);
    const ViewD& vw = *vwp;
    if (!__any_sync(FULL, wb.inimg)) continue;
    const float4* __restrict__ nrm = surv_normals<NRM>(B, vw);
    FwdState S = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0, 0, !wb.inimg, 0, nullptr};
    if (B->frag && wb.inimg)
      S.fl = B->frag + (vw.pix_base + (long long)wb.py * vw.W + wb.px) * (long long)fcap;
    if (four) {
      fwd_walk<NRM, 4, CNT>(B, wb, vals, rec, nrm, rg.x, rg.y, ts, TILE * TILE, pure, cap, skip,
                            eps, st[wid], sidx[wid], sslot[wid], fcap, S);
      // the pixel's sums over its four lanes
      S.C0 = pix_sum<4>(S.C0);
      S.C1 = pix_sum<4>(S.C1);
      S.C2 = pix_sum<4>(S.C2);
      S.D = pix_sum<4>(S.D);
      if constexpr (NRM) {
        S.N0 = pix_sum<4>(S.N0);
        S.N1 = pix_sum<4>(S.N1);
        S.N2 = pix_sum<4>(S.N2);
      }
      S.nfrag = pix_sum_i<4>(S.nfrag);
      S.last = pix_max_i<4>(S.last);
      if (wb.inimg && (threadIdx.x & 3) == 0) store_pixel<NRM>(B, vw, wb, S, image, alpha, depth, normal);
      // the tile's largest blended index: the backward skips the segments past it
      const unsigned ml = __reduce_max_sync(FULL, (unsigned)S.last);
      if ((threadIdx.x & 31) == 0 && ml > 0u) atomicMax(B->tile_last + wb.gt, (int)ml);
      if (fcap > 0) list_pixel(B, vw, wb, S.nb, fcap, (threadIdx.x & 3) == 0);
    } else {
      fwd_walk<NRM, 1, CNT>(B, wb, vals, rec, nrm, rg.x, rg.y, ts, TILE * TILE, pure, cap, skip,
                            eps, st[wid], sidx[wid], sslot[wid], fcap, S);
      if (wb.inimg) store_pixel<NRM>(B, vw, wb, S, image, alpha, depth, normal);
      if (fcap > 0) list_pixel(B, vw, wb, S.nb, fcap, true);
    }
  }
  queue_done(&c->work_fwd, &c->done_fwd);
}

// ---------------------------------------------------------------------------
// Resort window (Sec. 3.3).  Per pixel, fragments that pass the cap and skip
// tests enter a window of at most N_w (kept in registers) sorted by the depth
// of the chord's entry point, ties keeping arrival order; when it holds more
// than N_w fragments the nearest leaves it and is blended (stop-before-T<eps
// applies in this order); at the end of the list the rest leave nearest
// first.  The entry depth is zbar / rho_in (the record's reference depth is
// the tet's mean depth).
// ---------------------------------------------------------------------------
constexpr int WIN_MAX = 8;

struct Win {
  float k[WIN_MAX];
  float a[WIN_MAX];
  unsigned sl[WIN_MAX];
  int n;
};

__device__ __forceinline__ void win_insert(Win& w, float key, float a, unsigned slot) {
  int pos = 0;
#pragma unroll
  for (int i = 0; i < WIN_MAX; ++i) pos += (i < w.n) & (w.k[i] <= key);
#pragma unroll
  for (int i = WIN_MAX - 1; i > 0; --i) {
    if (i > pos && i <= w.n) {
      w.k[i] = w.k[i - 1];
      w.a[i] = w.a[i - 1];
      w.sl[i] = w.sl[i - 1];
    }
  }
#pragma unroll
  for (int i = 0; i < WIN_MAX; ++i) {
    if (i == pos) {
      w.k[i] = key;
      w.a[i] = a;
      w.sl[i] = slot;
    }
  }
  ++w.n;
}

__device__ __forceinline__ void win_pop(Win& w) {
#pragma unroll
  for (int i = 0; i < WIN_MAX - 1; ++i) {
    w.k[i] = w.k[i + 1];
    w.a[i] = w.a[i + 1];
    w.sl[i] = w.sl[i + 1];
  }
  --w.n;
}

// Blend one fragment leaving the window (forward).
template <bool NRM>
__device__ __forceinline__ void win_emit_fwd(const float4* __restrict__ rec,
                                             const float4* __restrict__ nrm, unsigned slot, float a,
                                             bool pure, float eps, float& T, float& C0, float& C1,
                                             float& C2, float& D, float& N0, float& N1, float& N2,
                                             bool& done) {
  const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
  if (!pure && Tn < eps) {
    done = true;
    return;
  }
  const float4 q5 = __ldg(rec + (size_t)slot * REC_Q + 5);
  const float wgt = __fmul_rn(T, a);
  C0 = __fmaf_rn(wgt, q5.y, C0);
  C1 = __fmaf_rn(wgt, q5.z, C1);
  C2 = __fmaf_rn(wgt, q5.w, C2);
  D = __fmaf_rn(wgt, q5.x, D);
  if constexpr (NRM) {
    const float4 n = __ldg(nrm + slot);
    N0 = __fmaf_rn(wgt, n.x, N0);
    N1 = __fmaf_rn(wgt, n.y, N1);
    N2 = __fmaf_rn(wgt, n.z, N2);
  }
  T = Tn;
}

template <int TILE, bool NRM>
__global__ void __launch_bounds__(WPB * 32) k_blend_fwd_win(const Batch* __restrict__ B,
                                                           float* __restrict__ image,
                                                           float* __restrict__ alpha,
                                                           float* __restrict__ depth,
                                                           float* __restrict__ normal) {
  pdl_wait();
  pdl_launch_dependents();
  constexpr int SB = (TILE / 8) * (TILE / 4);
  __shared__ float4 st[WPB][REC_Q][32];
  __shared__ unsigned sslot[WPB][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned ltm = (1u << lane) - 1u;
  Counters* c = B->ctr;
  const unsigned* __restrict__ vals = B->vals;
  const float4* __restrict__ rec = B->rec;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap, skip = B->alpha_skip, eps = B->t_eps;
  const int nw = B->resort_window;
  const int total = c->n_units * SB;
  for (int item = next_item(&c->work_fwd); item < total; item = next_item(&c->work_fwd)) {
    WarpBlock wb;
    const ViewD& vw = decode_item<TILE>(B, B->worklist, item, wb);
    if (!__any_sync(FULL, wb.inimg)) continue;
    const int2 rg = B->ranges[wb.gt];
    const float4* __restrict__ nrm = surv_normals<NRM>(B, vw);
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f;
    int nfrag = 0;
    bool done = !wb.inimg;
    Win win;
    win.n = 0;
    for (int g = rg.x; g < rg.y; g += 32) {
      if (!wb.cull_to(!done)) break;
      const int idx = g + lane;
      bool ov = false;
      unsigned slot = 0u;
      float4 q0;
      if (idx < rg.y) {
        slot = vals[idx];
        q0 = __ldg(rec + (size_t)slot * REC_Q);
        ov = !wb.misses(q0);
      }
      const unsigned m = __ballot_sync(FULL, ov);
      if (m == 0u) continue;
      if (ov) {
        const int pos = __popc(m & ltm);
        const float4* r = rec + (size_t)slot * REC_Q;
        st[wid][0][pos] = q0;
#pragma unroll
        for (int q = 1; q < REC_Q; ++q) st[wid][q][pos] = __ldg(r + q);
        sslot[wid][pos] = slot;
      }
      __syncwarp();
      const int cnt = __popc(m);
      for (int k = 0; k < cnt; ++k) {
        if (!done) {
          const Chord ch = chord_eval(st[wid][0][k], st[wid][1][k], st[wid][2][k], st[wid][3][k],
                                      wb.fpx, wb.fpy);
          if (ch.hit) {
            ++nfrag;
            const Opacity o = opacity_eval(st[wid][4][k], ch);
            const float a = pure ? o.alpha : fminf(o.alpha, cap);
            if (pure ? (a > 0.f) : (a >= skip)) {
              const float key = __fmul_rn(st[wid][5][k].x, __fmul_rn(o.rho_out, o.r));
              win_insert(win, key, a, sslot[wid][k]);
              if (win.n > nw) {
                const unsigned s0 = win.sl[0];
                const float a0 = win.a[0];
                win_pop(win);
                win_emit_fwd<NRM>(rec, nrm, s0, a0, pure, eps, T, C0, C1, C2, D, N0, N1, N2, done);
              }
            }
          }
        }
        if (__all_sync(FULL, done)) break;
      }
      __syncwarp();
    }
    // flush what is left in the window, nearest first
    while (!done && win.n > 0) {
      const unsigned s0 = win.sl[0];
      const float a0 = win.a[0];
      win_pop(win);
      win_emit_fwd<NRM>(rec, nrm, s0, a0, pure, eps, T, C0, C1, C2, D, N0, N1, N2, done);
    }
    if (wb.inimg) {
      const long long HW = (long long)vw.W * vw.H;
      const long long p = (long long)wb.py * vw.W + wb.px;
      image[3 * vw.pix_base + p] = C0;
      image[3 * vw.pix_base + HW + p] = C1;
      image[3 * vw.pix_base + 2 * HW + p] = C2;
      alpha[vw.pix_base + p] = 1.f - T;
      depth[vw.pix_base + p] = D;
      B->pix_T[vw.pix_base + p] = T;
      B->pix_last[vw.pix_base + p] = rg.y - rg.x;
      B->pix_nfrag[vw.pix_base + p] = nfrag;
      B->pix_CD[vw.pix_base + p] = make_float4(C0, C1, C2, D);
      if constexpr (NRM) store_normal(B, vw, p, normal, N0, N1, N2);
    }
  }
  queue_done(&c->work_fwd, &c->done_fwd);
}


// ---------------------------------------------------------------------------
// K7: backward blend.  Same warp blocks; each warp re-walks its tile's list
// back to front from the last entry any of its pixels blended, recomputes
// every fragment bit for bit, and accumulates the record-field gradients
// (per contributing lane, one vector atomic per field group) into the
// per-slot record gradient buffer.
// ---------------------------------------------------------------------------
template <int TILE, bool NRM, int NW, bool CNT = false>
__global__ void __launch_bounds__(NW * 32) k_blend_bwd(const Batch* __restrict__ B,
                                                      const float* __restrict__ dimage,
                                                      const float* __restrict__ dalpha,
                                                      const float* __restrict__ ddepth,
                                                      const float* __restrict__ dnormal,
                                                       GradOut zg) {
  pdl_wait();
  pdl_launch_dependents();
  constexpr int SB = (TILE / 8) * (TILE / 4);
  __shared__ float4 st[NW][REC_Q + NRM][32];
  __shared__ int sidx[NW][32];
  __shared__ unsigned sslot[NW][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned ltm = (1u << lane) - 1u;
  Counters* c = B->ctr;
  const unsigned* __restrict__ vals = B->vals;
  const float4* __restrict__ rec = B->rec;
  float4* __restrict__ rgrad = B->rec_grad;
  unsigned char* __restrict__ touched = B->rec_touched;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap, skip = B->alpha_skip;
  const int total = c->n_units_b * SB;
  const int fcap = B->frag_cap;
  constexpr bool count = CNT;   // TTS_FLAG_COUNT: an instantiation of its own
  // with per-pixel fragment lists and no pixel past the cap, nothing is left
  // for the list walk (its queue is not even taken)
  const bool walk = fcap == 0 || *reinterpret_cast<const volatile unsigned*>(&c->ovf_any) != 0u;
  for (int item = walk ? next_item(&c->work_bwd) : total; item < total;
       item = next_item(&c->work_bwd)) {
    WarpBlock wb;
    const ViewD& vw = decode_item<TILE>(B, B->worklist_b, item, wb);
    // with per-pixel fragment lists, only tiles holding a pixel past the cap
    // are walked here (their other pixels are left to k_blend_bwd_px)
    if (fcap > 0 && B->tile_ovf[wb.gt] == 0) continue;
    // a segment past every entry the tile's pixels blended has no work
    const int2 ts = B->tseg[wb.gt];
    if (ts.y > 1 && wb.seg * B->seg_len >= B->tile_last[wb.gt]) continue;
    const int2 rg = B->ranges[wb.gt];
    const long long HW = (long long)vw.W * vw.H;
    const long long p = (long long)wb.py * vw.W + wb.px;
    const float4* __restrict__ nrm = surv_normals<NRM>(B, vw);
    float Tfin = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gO = 0.f, gD = 0.f;
    float gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
    int last = 0;
    if (wb.inimg) {
      Tfin = B->pix_T[vw.pix_base + p];
      last = B->pix_last[vw.pix_base + p];
      if (fcap > 0 && B->pix_nb[vw.pix_base + p] <= fcap) last = 0;   // a listed pixel
      gC0 = dimage[3 * vw.pix_base + p];
      gC1 = dimage[3 * vw.pix_base + HW + p];
      gC2 = dimage[3 * vw.pix_base + 2 * HW + p];
      if (dalpha) gO = dalpha[vw.pix_base + p];
      if (ddepth) gD = ddepth[vw.pix_base + p];
      if (NRM && dnormal) {
        gN0 = dnormal[3 * vw.pix_base + p];
        gN1 = dnormal[3 * vw.pix_base + HW + p];
        gN2 = dnormal[3 * vw.pix_base + 2 * HW + p];
      }
    }
    // the list range of this item: the whole list, or one segment of a split
    // one; T and the suffix S start at the range's end
    int lo = rg.x, hi = rg.y;
    float T = Tfin, S = 0.f;
    if (ts.y > 1) {
      lo = rg.x + wb.seg * B->seg_len;
      hi = min(lo + B->seg_len, rg.y);
      if (wb.inimg && last > hi - rg.x) {
        // the pixel blends past this segment: T and the colour / depth /
        // normal at its end were stored by the forward; the suffix after it
        // is S = W - (gC.C + gD.D + gN.N at the end), W the same of the
        // final pixel
        const long long pj = ((long long)ts.x + wb.seg) * (TILE * TILE) + wb.tpix;
        const float4 a = __ldcg(B->pseg_a + pj);
        const float4 b4 = __ldcg(B->pseg_b + pj);
        float P = gC0 * a.y + gC1 * a.z + gC2 * a.w + gD * b4.x;
        if constexpr (NRM) P += gN0 * b4.y + gN1 * b4.z + gN2 * b4.w;
        const float4 cd = B->pix_CD[vw.pix_base + p];
        float W = gC0 * cd.x + gC1 * cd.y + gC2 * cd.z + gD * cd.w;
        if constexpr (NRM) {
          if (dnormal) {
            const float4 nf = B->pix_N[vw.pix_base + p];
            W += gN0 * nf.x + gN1 * nf.y + gN2 * nf.z;
          }
        }
        T = a.x;
        S = W - P;
      }
    }
    int maxlast = min(last, hi - rg.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxlast = max(maxlast, __shfl_xor_sync(FULL, maxlast, o));
    if (maxlast <= lo - rg.x) continue;
    const float gOT = gO * Tfin;
    const int top = rg.x + maxlast;
    // one group of lookahead on (slot, bbox), as in the forward: the group
    // [max(lo, ge - 32), ge) is tested while the next one's bboxes load
    int idx = max(lo, top - 32) + lane;
    unsigned slot = (idx < top) ? vals[idx] : 0u;
    float4 q0 = (idx < top) ? __ldg(rec + (size_t)slot * REC_Q) : make_float4(0.f, 0.f, -1.f, -1.f);
    int idn = max(lo, top - 64) + lane;
    unsigned slot_n = (idn < top - 32) ? vals[idn] : 0u;
    for (int ge = top; ge > lo; ge -= 32) {
      const int g0 = max(lo, ge - 32);
      const int idnn = max(lo, ge - 96) + lane;
      const float4 q0_n = (idn < ge - 32) ? __ldg(rec + (size_t)slot_n * REC_Q)
                                          : make_float4(0.f, 0.f, -1.f, -1.f);
      const unsigned slot_nn = (idnn < ge - 64) ? vals[idnn] : 0u;
      const bool live = wb.cull_to(last > g0 - rg.x);
      const bool ov = live && (idx < ge) && !wb.misses(q0);
      const unsigned m = __ballot_sync(FULL, ov);
      if (count && lane == 0) {
        atomicAdd(c->walk + 3, 1ull);
        atomicAdd(c->walk + 4, (unsigned long long)__popc(m));
      }
      if (m != 0u) {
      if (ov) {
        const int pos = __popc(m & ltm);
        const float4* r = rec + (size_t)slot * REC_Q;
        st[wid][0][pos] = q0;
#pragma unroll
        for (int q = 1; q < REC_Q; ++q) st[wid][q][pos] = __ldg(r + q);
        if constexpr (NRM) st[wid][REC_Q][pos] = __ldg(nrm + slot);
        sidx[wid][pos] = lane;
        sslot[wid][pos] = slot;
      }
      __syncwarp();
      for (int k = __popc(m) - 1; k >= 0; --k) {
        // some lane is active for every staged entry (they all lie below the
        // largest `last` of the warp)
        const bool active = (g0 + sidx[wid][k] - rg.x) < last;
        const Chord ch = chord_eval(st[wid][0][k], st[wid][1][k], st[wid][2][k], st[wid][3][k],
                                    wb.fpx, wb.fpy);
        bool contrib = active & ch.hit;
        Opacity o;
        float a = 0.f;
        if (contrib) {
          o = opacity_eval(st[wid][4][k], ch);
          a = pure ? o.alpha : fminf(o.alpha, cap);
          contrib = pure ? (a > 0.f) : (a >= skip);
        }
        float dpin = 0.f, dpout = 0.f;
        float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float gz = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
        float gn0 = 0.f, gn1 = 0.f, gn2 = 0.f;
        if (contrib) {
          const float4 q5 = st[wid][5][k];
          const float om = __fsub_rn(1.f, a);
          const float iom = rcp_approx(om);   // a <= cap < 1 (or a pure-mode alpha < 1)
          const float Ti = T * iom;
          float wv = gC0 * q5.y + gC1 * q5.z + gC2 * q5.w + gD * q5.x;
          if constexpr (NRM) {
            const float4 n = st[wid][REC_Q][k];
            wv += gN0 * n.x + gN1 * n.y + gN2 * n.z;
          }
          const float dLda = Ti * wv - (S - gOT) * iom;
          S += Ti * a * wv;
          T = Ti;
          const float wgt = Ti * a;
          gz = wgt * gD;
          gc0 = wgt * gC0;
          gc1 = wgt * gC1;
          gc2 = wgt * gC2;
          gn0 = wgt * gN0;
          gn1 = wgt * gN1;
          gn2 = wgt * gN2;
          const bool clamped = !pure && (o.alpha > cap);
          if (!clamped) {
            // alpha = (1 - e1) B with x = s (f_prev - f_next), y = s f_next
            const float dx = dLda * o.e1 * o.B;
            const float dy = -dLda * o.alpha * (1.f - o.B);
            const float iin = o.rho_out * o.r, iout = o.rho_in * o.r;
            dpin = -dx * o.sGz * iin * iin;
            dpout = (dx - dy) * o.sGz * iout * iout;
            const float dsGz = dx * (ch.p_out - ch.p_in) * o.r - dy * ch.p_out * iout;
            r4 = make_float4(dy, dsGz, (dy + dsGz) * ch.dx, (dy + dsGz) * ch.dy);
          }
        }
        // each contributing lane adds its record-field gradients with vector
        // atomics (the few lanes of one candidate meet in L2)
        if (contrib) {
          const unsigned sl = sslot[wid][k];
          touched[sl] = 1;   // the same byte from every contributing lane
          add_frag_grad<NRM>(rgrad + (size_t)sl * REC_Q, ch.kin, ch.kout, dpin, dpout, ch.dx,
                             ch.dy, r4, make_float4(gz, gc0, gc1, gc2), gn0, gn1, gn2);
        }
      }
      __syncwarp();
      }
      idx = idn;
      slot = slot_n;
      q0 = q0_n;
      idn = idnn;
      slot_n = slot_nn;
    }
  }
  zero_tail(B, zg, &c->zero_q);
  queue_done(&c->work_bwd, &c->done_bwd, &c->zero_q);
}

// ---------------------------------------------------------------------------
// K7 from the per-pixel fragment lists.  Warps take the listed pixels (the
// forward's task list) in grid stride, one pixel per warp at a time and one
// lane per fragment, in chunks of 32 fragments from the pixel's last chunk
// to its first.  Each lane recomputes its fragment from its record bit for
// bit as the list walk does; the transmittance in front of each fragment is
// the product of (1 - alpha') of the fragments before it (a product scan over
// the lanes, times the product of the earlier chunks) and the suffix of
// T_j alpha'_j w_j behind it a sum scan (plus the later chunks' sums).  The
// record-field gradients leave as in the list walk, one set of vector
// atomics per fragment.  Pixels past the cap are left to k_blend_bwd.
// ---------------------------------------------------------------------------
constexpr int PXW = 4;          // warps per block
constexpr int PX_CHUNKS = 8;    // 32-fragment chunks of a pixel (frag_cap <= 255)

// Fragment i of a pixel: its record slot, chord, opacity and alpha'.
struct PxFrag {
  unsigned sl;
  float4 q5;
  Chord ch;
  Opacity o;
  float a;
};

__device__ __forceinline__ void px_frag(const float4* __restrict__ rec, const unsigned* fl, int i,
                                        bool pure, float cap, float fpx, float fpy, PxFrag& F) {
  F.sl = fl[i];
  const float4* r = rec + (size_t)F.sl * REC_Q;
  const float4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2), q3 = __ldg(r + 3);
  const float4 q4 = __ldg(r + 4);
  F.q5 = __ldg(r + 5);
  F.ch = chord_eval(q0, q1, q2, q3, fpx, fpy);
  F.o = opacity_eval(q4, F.ch);
  F.a = pure ? F.o.alpha : fminf(F.o.alpha, cap);
}

// Product of x over the lanes below (exclusive; 1 at lane 0) and over all lanes.
__device__ __forceinline__ float prod_excl(float x, float* all) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x = __fmul_rn(y, x);
  }
  *all = __shfl_sync(FULL, x, 31);
  const float e = __shfl_up_sync(FULL, x, 1);
  return lane == 0 ? 1.f : e;
}

// Sum of x over the lanes above (exclusive; 0 at lane 31) and over all lanes.
__device__ __forceinline__ float sum_above(float x, float* all) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float y = __shfl_down_sync(FULL, x, d);
    if (lane + d < 32) x += y;
  }
  *all = __shfl_sync(FULL, x, 0);
  const float e = __shfl_down_sync(FULL, x, 1);
  return lane == 31 ? 0.f : e;
}

template <int TILE, bool NRM>
__global__ void __launch_bounds__(PXW * 32) k_blend_bwd_px(const Batch* __restrict__ B,
                                                           const float* __restrict__ dimage,
                                                           const float* __restrict__ dalpha,
                                                           const float* __restrict__ ddepth,
                                                           const float* __restrict__ dnormal,
                                                           GradOut zg) {
  pdl_wait();
  pdl_launch_dependents();
  Counters* c = B->ctr;
  const int lane = threadIdx.x & 31;
  const unsigned n = c->px_n;
  const int fcap = B->frag_cap;
  const float4* __restrict__ rec = B->rec;
  float4* __restrict__ rgrad = B->rec_grad;
  unsigned char* __restrict__ touched = B->rec_touched;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap;
  const unsigned stride = gridDim.x * PXW;
  unsigned t = blockIdx.x * PXW + (threadIdx.x >> 5);
  uint2 task = (t < n) ? B->px_list[t] : make_uint2(0u, 0u);
  for (; t < n; t += stride) {
    const long long pg = task.x;
    const int nb = (int)(task.y & 0xffu);
    const ViewD& vw = B->vw[task.y >> 8];
    if (t + stride < n) task = B->px_list[t + stride];   // the next task's entry, early
    const long long p = pg - vw.pix_base;
    const int py = (int)(p / vw.W), px = (int)(p - (long long)py * vw.W);
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const float4* __restrict__ nrm = surv_normals<NRM>(B, vw);
    const long long HW = (long long)vw.W * vw.H;
    const float Tfin = B->pix_T[pg];
    const float gC0 = dimage[3 * vw.pix_base + p];
    const float gC1 = dimage[3 * vw.pix_base + HW + p];
    const float gC2 = dimage[3 * vw.pix_base + 2 * HW + p];
    const float gO = dalpha ? dalpha[pg] : 0.f;
    const float gD = ddepth ? ddepth[pg] : 0.f;
    float gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
    if (NRM && dnormal) {
      gN0 = dnormal[3 * vw.pix_base + p];
      gN1 = dnormal[3 * vw.pix_base + HW + p];
      gN2 = dnormal[3 * vw.pix_base + 2 * HW + p];
    }
    const float gOT = gO * Tfin;
    const unsigned* __restrict__ fl = B->frag + pg * (long long)fcap;
    const int nch = (nb + 31) >> 5;
    // the transmittance in front of each chunk (more than one chunk: a first
    // pass over the earlier chunks' alpha')
    float Tch[PX_CHUNKS];
    Tch[0] = 1.f;
#pragma unroll
    for (int k = 1; k < PX_CHUNKS; ++k) {
      Tch[k] = Tch[k - 1];
      if (k < nch) {
        const int i = 32 * (k - 1) + lane;
        float om = 1.f;
        if (i < nb) {
          PxFrag F;
          px_frag(rec, fl, i, pure, cap, fpx, fpy, F);
          om = __fsub_rn(1.f, F.a);
        }
        float all;
        prod_excl(om, &all);
        Tch[k] = __fmul_rn(Tch[k - 1], all);
      }
    }
    float Sc = 0.f;   // suffix of the later chunks
#pragma unroll 1
    for (int k = nch - 1; k >= 0; --k) {
      float T0 = Tch[0];
#pragma unroll
      for (int q = 1; q < PX_CHUNKS; ++q)
        if (q == k) T0 = Tch[q];
      const int i = 32 * k + lane;
      const bool on = i < nb;
      PxFrag F;
      float om = 1.f, wv = 0.f;
      float4 nv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (on) {
        px_frag(rec, fl, i, pure, cap, fpx, fpy, F);
        om = __fsub_rn(1.f, F.a);
        wv = gC0 * F.q5.y + gC1 * F.q5.z + gC2 * F.q5.w + gD * F.q5.x;
        if constexpr (NRM) {
          nv = __ldg(nrm + F.sl);
          wv += gN0 * nv.x + gN1 * nv.y + gN2 * nv.z;
        }
      }
      float pall, sall;
      const float Ti = __fmul_rn(T0, prod_excl(om, &pall));
      const float cterm = on ? Ti * F.a * wv : 0.f;
      const float S = Sc + sum_above(cterm, &sall);
      Sc += sall;
      if (on) {
        const float iom = rcp_approx(om);
        const float dLda = Ti * wv - (S - gOT) * iom;
        const float wgt = Ti * F.a;
        const Chord& ch = F.ch;
        const Opacity& o = F.o;
        float dpin = 0.f, dpout = 0.f;
        float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool clamped = !pure && (o.alpha > cap);
        if (!clamped) {
          const float dx = dLda * o.e1 * o.B;
          const float dy = -dLda * o.alpha * (1.f - o.B);
          const float iin = o.rho_out * o.r, iout = o.rho_in * o.r;
          dpin = -dx * o.sGz * iin * iin;
          dpout = (dx - dy) * o.sGz * iout * iout;
          const float dsGz = dx * (ch.p_out - ch.p_in) * o.r - dy * ch.p_out * iout;
          r4 = make_float4(dy, dsGz, (dy + dsGz) * ch.dx, (dy + dsGz) * ch.dy);
        }
        touched[F.sl] = 1;
        add_frag_grad<NRM>(rgrad + (size_t)F.sl * REC_Q, ch.kin, ch.kout, dpin, dpout, ch.dx, ch.dy,
                           r4, make_float4(wgt * gD, wgt * gC0, wgt * gC1, wgt * gC2), wgt * gN0,
                           wgt * gN1, wgt * gN2);
      }
    }
  }
  // the vertex-gradient arrays of the scatter that follows, cleared by the
  // warps once their pixels are done (the list walk takes what is left)
  zero_tail(B, zg, &c->zero_q);
}

// Backward with the resort window: replays the forward (same walk, same
// window, same stop) front to back.  With W = gC.C + gD.D of the final pixel
// and the running prefix P of T_j a_j w_j, the suffix of fragment i is
// W - P - T_i a_i w_i, so dL/da_i = T_i w_i - (suffix - gO T_final)/(1 - a_i).
// Each emitted fragment's record is reloaded and its chord recomputed; the
// record-field gradients leave as per-lane vector atomics.
template <int TILE, bool NRM>
__global__ void __launch_bounds__(WPB * 32) k_blend_bwd_win(const Batch* __restrict__ B,
                                                           const float* __restrict__ dimage,
                                                           const float* __restrict__ dalpha,
                                                           const float* __restrict__ ddepth,
                                                           const float* __restrict__ dnormal,
                                                            GradOut zg) {
  pdl_wait();
  pdl_launch_dependents();
  constexpr int SB = (TILE / 8) * (TILE / 4);
  __shared__ float4 st[WPB][REC_Q][32];
  __shared__ unsigned sslot[WPB][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned ltm = (1u << lane) - 1u;
  Counters* c = B->ctr;
  const unsigned* __restrict__ vals = B->vals;
  const float4* __restrict__ rec = B->rec;
  float4* __restrict__ rgrad = B->rec_grad;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap, skip = B->alpha_skip, eps = B->t_eps;
  const int nw = B->resort_window;
  const int total = c->n_units_b * SB;
  for (int item = next_item(&c->work_bwd); item < total; item = next_item(&c->work_bwd)) {
    WarpBlock wb;
    const ViewD& vw = decode_item<TILE>(B, B->worklist_b, item, wb);
    if (!__any_sync(FULL, wb.inimg)) continue;
    const int2 rg = B->ranges[wb.gt];
    const long long HW = (long long)vw.W * vw.H;
    const long long pp = (long long)wb.py * vw.W + wb.px;
    const float4* __restrict__ nrm = surv_normals<NRM>(B, vw);
    float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gO = 0.f, gD = 0.f, Tfin = 1.f, Wt = 0.f;
    float gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
    if (wb.inimg) {
      Tfin = B->pix_T[vw.pix_base + pp];
      gC0 = dimage[3 * vw.pix_base + pp];
      gC1 = dimage[3 * vw.pix_base + HW + pp];
      gC2 = dimage[3 * vw.pix_base + 2 * HW + pp];
      if (dalpha) gO = dalpha[vw.pix_base + pp];
      if (ddepth) gD = ddepth[vw.pix_base + pp];
      const float4 cd = B->pix_CD[vw.pix_base + pp];
      Wt = gC0 * cd.x + gC1 * cd.y + gC2 * cd.z + gD * cd.w;
      if (NRM && dnormal) {
        gN0 = dnormal[3 * vw.pix_base + pp];
        gN1 = dnormal[3 * vw.pix_base + HW + pp];
        gN2 = dnormal[3 * vw.pix_base + 2 * HW + pp];
        const float4 nf = B->pix_N[vw.pix_base + pp];
        Wt += gN0 * nf.x + gN1 * nf.y + gN2 * nf.z;
      }
    }
    const float gOT = gO * Tfin;
    float T = 1.f, Pw = 0.f;
    bool done = !wb.inimg;
    Win win;
    win.n = 0;
    // adjoint of one fragment leaving the window
    auto emit = [&](unsigned slot, float a) {
      const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
      if (!pure && Tn < eps) {
        done = true;
        return;
      }
      const float4* r = rec + (size_t)slot * REC_Q;
      const float4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2), q3 = __ldg(r + 3);
      const float4 q4 = __ldg(r + 4), q5 = __ldg(r + 5);
      const Chord ch = chord_eval(q0, q1, q2, q3, wb.fpx, wb.fpy);
      const Opacity o = opacity_eval(q4, ch);
      float wv = gC0 * q5.y + gC1 * q5.z + gC2 * q5.w + gD * q5.x;
      float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (NRM) {
        n = __ldg(nrm + slot);
        wv += gN0 * n.x + gN1 * n.y + gN2 * n.z;
      }
      const float twa = T * a * wv;
      const float suffix = Wt - Pw - twa;
      const float dLda = T * wv - (suffix - gOT) * rcp_approx(__fsub_rn(1.f, a));
      Pw += twa;
      const float wgt = T * a;
      B->rec_touched[slot] = 1;
      const bool clamped = !pure && (o.alpha > cap);
      float dpin = 0.f, dpout = 0.f;
      float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!clamped) {
        const float dx = dLda * o.e1 * o.B;
        const float dy = -dLda * o.alpha * (1.f - o.B);
        const float iin = o.rho_out * o.r, iout = o.rho_in * o.r;
        dpin = -dx * o.sGz * iin * iin;
        dpout = (dx - dy) * o.sGz * iout * iout;
        const float dsGz = dx * (ch.p_out - ch.p_in) * o.r - dy * ch.p_out * iout;
        r4 = make_float4(dy, dsGz, (dy + dsGz) * ch.dx, (dy + dsGz) * ch.dy);
      }
      add_frag_grad<NRM>(rgrad + (size_t)slot * REC_Q, ch.kin, ch.kout, dpin, dpout, ch.dx, ch.dy,
                         r4, make_float4(wgt * gD, wgt * gC0, wgt * gC1, wgt * gC2), wgt * gN0,
                         wgt * gN1, wgt * gN2);
      T = Tn;
    };
    for (int g = rg.x; g < rg.y; g += 32) {
      if (!wb.cull_to(!done)) break;
      const int idx = g + lane;
      bool ov = false;
      unsigned slot = 0u;
      float4 q0;
      if (idx < rg.y) {
        slot = vals[idx];
        q0 = __ldg(rec + (size_t)slot * REC_Q);
        ov = !wb.misses(q0);
      }
      const unsigned m = __ballot_sync(FULL, ov);
      if (m == 0u) continue;
      if (ov) {
        const int pos = __popc(m & ltm);
        const float4* r = rec + (size_t)slot * REC_Q;
        st[wid][0][pos] = q0;
#pragma unroll
        for (int q = 1; q < REC_Q; ++q) st[wid][q][pos] = __ldg(r + q);
        sslot[wid][pos] = slot;
      }
      __syncwarp();
      const int cnt = __popc(m);
      for (int k = 0; k < cnt; ++k) {
        if (!done) {
          const Chord ch = chord_eval(st[wid][0][k], st[wid][1][k], st[wid][2][k], st[wid][3][k],
                                      wb.fpx, wb.fpy);
          if (ch.hit) {
            const Opacity o = opacity_eval(st[wid][4][k], ch);
            const float a = pure ? o.alpha : fminf(o.alpha, cap);
            if (pure ? (a > 0.f) : (a >= skip)) {
              const float key = __fmul_rn(st[wid][5][k].x, __fmul_rn(o.rho_out, o.r));
              win_insert(win, key, a, sslot[wid][k]);
              if (win.n > nw) {
                const unsigned s0 = win.sl[0];
                const float a0 = win.a[0];
                win_pop(win);
                emit(s0, a0);
              }
            }
          }
        }
        if (__all_sync(FULL, done)) break;
      }
      __syncwarp();
    }
    while (!done && win.n > 0) {
      const unsigned s0 = win.sl[0];
      const float a0 = win.a[0];
      win_pop(win);
      emit(s0, a0);
    }
  }
  zero_tail(B, zg, &c->zero_q);
  queue_done(&c->work_bwd, &c->done_bwd, &c->zero_q);
}

// ---------------------------------------------------------------------------
// K8: record -> vertex adjoint.  Only the (survivor, view) slots the blend
// backward touched carry a gradient (a sixth of them on a typical step), so
// the slots are compacted first: each warp takes 32 survivors at a time,
// reads their touched flags (eight views at a time) and appends the touched
// (survivor, view) pairs to a queue of its own in shared memory; every 32
// queued pairs are then processed one per lane.  A lane recomputes the
// view's tet geometry, applies the adjoint of the record fields (App. A.3's
// affine SDF and the face planes) and clears the slot's gradient and flag.
// A survivor's pairs sit in consecutive lanes; they are summed over those
// lanes and the first of them scatters the sum into dV, df, drgb.
// The reference point x_r (ray through the bbox corner pixel at the centroid
// depth) is held constant: the fragment opacity does not depend on it.
// With the normal map channel, the per-view dL/dn (record gradient .w of the
// face rows) is summed over the survivor's lanes and pushed once through the
// world-space n = g / |g| of the tet's affine SDF.
// ---------------------------------------------------------------------------
constexpr int TB_WARPS = 4;
constexpr int TB_QUEUE = 512;   // ring of (survivor, view) pairs per warp (> 31 + 32 * 8)

template <bool NRM>
__global__ void __launch_bounds__(TB_WARPS * 32, 4) k_tet_bwd(const Batch* __restrict__ B,
                                                              GradOut go) {
  pdl_wait();
  pdl_launch_dependents();
  __shared__ int2 s_q[TB_WARPS][TB_QUEUE];
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int nsurv = B->ctr->n_surv[s];
  const int nv = S.view_cnt;
  const float sv = B->s;
  float* __restrict__ gV = go.dV[s];
  float* __restrict__ gf = go.df[s];
  float* __restrict__ gc = go.drgb[s];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int2* __restrict__ q = s_q[wid];
  unsigned head = 0u, tail = 0u;   // warp-uniform ring positions

  // one (survivor, view) pair per lane (k < 0: none), then the per-survivor
  // sums and their scatter
  auto process = [&](int2 pr) {
    const int k = pr.x;
    float3 dv[4] = {f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0)};
    float dfv[4] = {0.f, 0.f, 0.f, 0.f};
    float3 dcol = f3(0, 0, 0);
    float3 dnw = f3(0, 0, 0);
    bool any = false;
    int4 t = make_int4(0, 0, 0, 0);
    TetIn in;
    if (k >= 0) {
      t = B->surv_T[S.surv_off + k];
      load_tet_ids<false>(S, t, in);
      const ViewD& vw = B->vw[B->scene_views[S.view_off + pr.y]];
      const long long slot = vw.rec_base + k;
      B->rec_touched[slot] = 0;
      do {
        // face-major rows: (dP, dA, dB, normal component) of faces 0..3, then
        // the opacity row and the depth / colour row
        float4* gq = B->rec_grad + slot * REC_Q;
        const float4 r0 = gq[0], r1 = gq[1], r2 = gq[2], r3 = gq[3], g4 = gq[4], g5 = gq[5];
        const float4 g0 = make_float4(r0.w, r1.w, r2.w, 0.f);
        const float4 g1 = make_float4(r0.x, r1.x, r2.x, r3.x);
        const float4 g2 = make_float4(r0.y, r1.y, r2.y, r3.y);
        const float4 g3 = make_float4(r0.z, r1.z, r2.z, r3.z);
        // the forward's pixel bbox corner, from the record: q0 = (+-(i0 + .5), +-(j0 + .5), ...)
        const float4 q0 = __ldg(B->rec + slot * REC_Q);
        const float mag = fabsf(g0.x) + fabsf(g0.y) + fabsf(g0.z) + fabsf(g1.x) + fabsf(g1.y) + fabsf(g1.z) + fabsf(g1.w) + fabsf(g2.x) +
                          fabsf(g2.y) + fabsf(g2.z) + fabsf(g2.w) + fabsf(g3.x) + fabsf(g3.y) +
                          fabsf(g3.z) + fabsf(g3.w) + fabsf(g4.x) + fabsf(g4.y) + fabsf(g4.z) +
                          fabsf(g4.w) + fabsf(g5.x) + fabsf(g5.y) + fabsf(g5.z) + fabsf(g5.w);
        if (mag == 0.f) break;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        gq[0] = z4; gq[1] = z4; gq[2] = z4; gq[3] = z4; gq[4] = z4; gq[5] = z4;
        dnw = dnw + f3(g0.x, g0.y, g0.z);
        Geo G;
        tet_geometry_at(vw, in, (int)(fabsf(q0.x) - 0.5f), (int)(fabsf(q0.y) - 0.5f), G);
        if (!G.visible) break;
        any = true;
        const float gPs[4] = {g1.x, g1.y, g1.z, g1.w};
        const float gAs[4] = {g2.x, g2.y, g2.z, g2.w};
        const float gBs[4] = {g3.x, g3.y, g3.z, g3.w};
        float3 dX[4] = {f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0)};
        float dff[4] = {0.f, 0.f, 0.f, 0.f};
        // All of the geometry lives in the pixel-scaled frame xi = (fx x, fy y, z)
        // where the record is P = m.x_r - 1, A = z_r m_x, B = z_r m_y with
        // m = n / e, F = s f(x_r), K0 = s z_r g.d_r, Kx = s z_r g_x, Ky = s z_r g_y.
        const float3 xr = G.zr * G.dr;
  #pragma unroll
        for (int fk = 0; fk < 4; ++fk) {
          const int sl = G.slot_of[fk];
          const float gP = (sl == 0) ? gPs[0] : (sl == 1) ? gPs[1] : (sl == 2) ? gPs[2] : gPs[3];
          const float gA = (sl == 0) ? gAs[0] : (sl == 1) ? gAs[1] : (sl == 2) ? gAs[2] : gAs[3];
          const float gB = (sl == 0) ? gBs[0] : (sl == 1) ? gBs[1] : (sl == 2) ? gBs[2] : gBs[3];
          const int i = kFaceVerts[fk][0], j = kFaceVerts[fk][1], l = kFaceVerts[fk][2];
          const float3 dm = f3(gP * xr.x + gA * G.zr, gP * xr.y + gB * G.zr, gP * xr.z);
          const float e = G.e[fk];
          const float3 n = G.n[fk];
          const float ie = rcp_approx(e);
          const float lam = dot3(n, dm) * (ie * ie);
          const float3 Xi = G.xm + G.y[i];
          const float3 dn = ie * dm - lam * Xi;
          dX[i] = dX[i] - lam * n;
          const float3 dnr = G.sgn[fk] * dn;
          const float3 ea = G.y[j] - G.y[i], eb = G.y[l] - G.y[i];
          const float3 da = cross3(eb, dnr), db = cross3(dnr, ea);
          dX[j] = dX[j] + da;
          dX[l] = dX[l] + db;
          dX[i] = dX[i] - (da + db);
        }
        const float dfr = sv * g4.x;
        float3 dg = f3(sv * G.zr * (g4.y * G.dr.x + g4.z), sv * G.zr * (g4.y * G.dr.y + g4.w),
                       sv * G.zr * g4.y);
        dg = dg + dfr * G.w;     // f_r = f_m + g.(x_r - x_m)
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          dff[q] += 0.25f * dfr;
          dX[q] = dX[q] - (0.25f * dfr) * G.g;
        }
        // g = Y^-1 df with Y rows y_j - y_0 (j = 1..3)
        const float idet = rcp_approx(G.det);
        const float dd1 = dot3(G.cof[0], dg) * idet, dd2 = dot3(G.cof[1], dg) * idet,
                    dd3 = dot3(G.cof[2], dg) * idet;
        dff[1] += dd1; dff[2] += dd2; dff[3] += dd3;
        dff[0] -= dd1 + dd2 + dd3;
        dX[1] = dX[1] - dd1 * G.g;
        dX[2] = dX[2] - dd2 * G.g;
        dX[3] = dX[3] - dd3 * G.g;
        dX[0] = dX[0] + (dd1 + dd2 + dd3) * G.g;
        // depth term: zbar = mean camera z (unscaled axis)
  #pragma unroll
        for (int q = 0; q < 4; ++q) dX[q].z += 0.25f * g5.x;
        // xi = S (R v + t), S = diag(fx, fy, 1)  ->  dv = R^T S dxi
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          dv[q] = dv[q] + rotT(vw.R, f3(vw.fx * dX[q].x, vw.fy * dX[q].y, dX[q].z));
          dfv[q] += dff[q];
        }
        dcol = dcol + f3(0.25f * g5.y, 0.25f * g5.z, 0.25f * g5.w);
      } while (0);
    }
    // sums over each run of lanes holding the same survivor and view group
    // (one survivor's pairs of one group of eight views: at most 8 lanes)
    const int kp = __shfl_up_sync(0xffffffffu, k, 1);
    const int gp = __shfl_up_sync(0xffffffffu, pr.y >> 3, 1);
    const bool run_head = lane == 0 || kp != k || gp != (pr.y >> 3);
    const unsigned heads = __ballot_sync(0xffffffffu, run_head);
    const int run = __popc(heads & (0xffffffffu >> (31 - lane)));   // run index of the lane
    float acc[22] = {dv[0].x, dv[0].y, dv[0].z, dv[1].x, dv[1].y, dv[1].z, dv[2].x, dv[2].y,
                     dv[2].z, dv[3].x, dv[3].y, dv[3].z, dfv[0], dfv[1], dfv[2], dfv[3],
                     dcol.x, dcol.y, dcol.z, dnw.x, dnw.y, dnw.z};
    int anyi = any ? 1 : 0;
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
      const int rd = __shfl_down_sync(0xffffffffu, run, d);
      const bool take = lane + d < 32 && rd == run;
#pragma unroll
      for (int j = 0; j < (NRM ? 22 : 19); ++j) {
        const float y = __shfl_down_sync(0xffffffffu, acc[j], d);
        if (take) acc[j] += y;
      }
      const int ya = __shfl_down_sync(0xffffffffu, anyi, d);
      if (take) anyi |= ya;
    }
    if (!run_head || k < 0) return;
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      dv[q4] = f3(acc[3 * q4], acc[3 * q4 + 1], acc[3 * q4 + 2]);
      dfv[q4] = acc[12 + q4];
    }
    dcol = f3(acc[16], acc[17], acc[18]);
    any = anyi != 0;
    if (NRM) {
      dnw = f3(acc[19], acc[20], acc[21]);
      if (dnw.x != 0.f || dnw.y != 0.f || dnw.z != 0.f) {
        TetGrad TG;
        tet_grad(in.v, in.f, TG);
        float ih, sg;
        const float3 n = tet_unit_normal(TG, &ih, &sg);
        if (ih > 0.f) {
          tet_grad_adjoint(TG, tet_normal_adjoint(n, ih, sg, dnw), 0.f, dv, dfv);
          any = true;
        }
      }
    }
    if (!any) return;
    const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      atomicAdd(gV + 3ll * id[q4], dv[q4].x);
      atomicAdd(gV + 3ll * id[q4] + 1, dv[q4].y);
      atomicAdd(gV + 3ll * id[q4] + 2, dv[q4].z);
      atomicAdd(gf + id[q4], dfv[q4]);
      atomicAdd(gc + 3ll * id[q4], dcol.x);
      atomicAdd(gc + 3ll * id[q4] + 1, dcol.y);
      atomicAdd(gc + 3ll * id[q4] + 2, dcol.z);
    }
  };

  const int gw = blockIdx.x * TB_WARPS + wid, nw = gridDim.x * TB_WARPS;
  for (int base = gw * 32; base < nsurv; base += nw * 32) {
    const int k = base + lane;
    for (int v0 = 0; v0 < nv; v0 += 8) {
      // the touched flags of eight views, loaded together
      unsigned m = 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (k < nsurv && v0 + j < nv)
          m |= (unsigned)(B->rec_touched[B->vw[B->scene_views[S.view_off + v0 + j]].rec_base + k] != 0)
               << j;
      const int c = __popc(m);
      int incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const unsigned tot = (unsigned)__shfl_sync(0xffffffffu, incl, 31);
      unsigned p = tail + (unsigned)(incl - c);
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        q[p++ & (TB_QUEUE - 1)] = make_int2(k, v0 + j);
      }
      tail += tot;
      __syncwarp();
      while (tail - head >= 32u) {
        const int2 pr = q[(head + lane) & (TB_QUEUE - 1)];
        __syncwarp();
        head += 32u;
        process(pr);
      }
    }
  }
  if (tail != head) {   // the last, partial batch
    const int2 pr = (head + lane < tail) ? q[(head + lane) & (TB_QUEUE - 1)] : make_int2(-1, 0);
    process(pr);
  }
}

// Clears dV, df, drgb of every scene before the record -> vertex scatter
// (16-byte stores where the arrays allow, grid-stride).  grid (blocks, n_scenes)
__global__ void __launch_bounds__(256) k_zero_grads(const Batch* __restrict__ B, GradOut go) {
  pdl_wait();
  pdl_launch_dependents();
  const int s = blockIdx.y;
  const long long N = B->sc[s].N;
  float* const arr[3] = {go.dV[s], go.df[s], go.drgb[s]};
  const long long len[3] = {3 * N, N, 3 * N};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int a = 0; a < 3; ++a) {
    float* p = arr[a];
    const long long n = len[a];
    // head up to 16-byte alignment, then float4 stores, then the tail
    const long long head = min(n, (long long)((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15) / 4);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < head; i += stride) p[i] = 0.f;
    float4* q = reinterpret_cast<float4*>(p + head);
    const long long n4 = (n - head) / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride)
      q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = head + 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
      p[i] = 0.f;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
static int occ_blocks(K kern, int threads, int sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess || per < 1)
    per = 4;
  return per * sms;
}

template <int TILE, bool NRM, int NW>
static void blend_grid_t(int sms, int window, int* fwd_blocks, int* bwd_blocks) {
  if (window > 0) {
    *fwd_blocks = occ_blocks(k_blend_fwd_win<TILE, NRM>, WPB * 32, sms);
    *bwd_blocks = occ_blocks(k_blend_bwd_win<TILE, NRM>, WPB * 32, sms);
  } else {
    *fwd_blocks = occ_blocks(k_blend_fwd<TILE, NRM, NW>, NW * 32, sms);
    *bwd_blocks = occ_blocks(k_blend_bwd<TILE, NRM, NW>, NW * 32, sms);
  }
}

// warps per block of the main blend kernels: 2, 4 or 8
static int warps_index(int warps) { return warps == 2 ? 0 : warps == 8 ? 2 : 1; }

template <int TILE, bool NRM>
static void blend_grid_w(int warps, int sms, int window, int* f, int* b) {
  switch (warps_index(warps)) {
    case 0: blend_grid_t<TILE, NRM, 2>(sms, window, f, b); break;
    case 2: blend_grid_t<TILE, NRM, 8>(sms, window, f, b); break;
    default: blend_grid_t<TILE, NRM, 4>(sms, window, f, b); break;
  }
}

void blend_grid(int tile, bool normals, int window, int warps, int sms, int* fwd_blocks,
                int* bwd_blocks) {
  static int cache[3][2][2][3][2] = {};
  const int ti = (tile == 8) ? 0 : (tile == 16) ? 1 : 2;
  const int ni = normals ? 1 : 0, wi = (window > 0) ? 1 : 0;
  int* c = cache[ti][ni][wi][warps_index(warps)];
  if (c[0] > 0) {
    *fwd_blocks = c[0];
    *bwd_blocks = c[1];
    return;
  }
  switch (tile * 2 + ni) {
    case 16: blend_grid_w<8, false>(warps, sms, window, fwd_blocks, bwd_blocks); break;
    case 17: blend_grid_w<8, true>(warps, sms, window, fwd_blocks, bwd_blocks); break;
    case 32: blend_grid_w<16, false>(warps, sms, window, fwd_blocks, bwd_blocks); break;
    case 33: blend_grid_w<16, true>(warps, sms, window, fwd_blocks, bwd_blocks); break;
    case 64: blend_grid_w<32, false>(warps, sms, window, fwd_blocks, bwd_blocks); break;
    default: blend_grid_w<32, true>(warps, sms, window, fwd_blocks, bwd_blocks); break;
  }
  c[0] = *fwd_blocks;
  c[1] = *bwd_blocks;
}

// Persistent grid of the pixel-list backward: as many blocks as fit at once.
int px_grid(int tile, bool normals, int sms) {
  static int cache[3][2] = {};
  const int ti = (tile == 8) ? 0 : (tile == 16) ? 1 : 2, ni = normals ? 1 : 0;
  if (cache[ti][ni] > 0) return cache[ti][ni];
  int g = 0;
  switch (tile * 2 + ni) {
    case 16: g = occ_blocks(k_blend_bwd_px<8, false>, PXW * 32, sms); break;
    case 17: g = occ_blocks(k_blend_bwd_px<8, true>, PXW * 32, sms); break;
    case 32: g = occ_blocks(k_blend_bwd_px<16, false>, PXW * 32, sms); break;
    case 33: g = occ_blocks(k_blend_bwd_px<16, true>, PXW * 32, sms); break;
    case 64: g = occ_blocks(k_blend_bwd_px<32, false>, PXW * 32, sms); break;
    default: g = occ_blocks(k_blend_bwd_px<32, true>, PXW * 32, sms); break;
  }
  cache[ti][ni] = g;
  return g;
}

template <int TILE, bool NRM, int NW>
static void fwd_nw(const HostPlan& P, const Batch* dB, float* image, float* alpha, float* depth,
                   float* normal, cudaStream_t st) {
  if (P.count)
    launch_k(k_blend_fwd<TILE, NRM, NW, true>, dim3(P.blend_fwd_blocks), dim3(NW * 32), 0, st, dB,
             image, alpha, depth, normal);
  else
    launch_k(k_blend_fwd<TILE, NRM, NW>, dim3(P.blend_fwd_blocks), dim3(NW * 32), 0, st, dB, image,
             alpha, depth, normal);
}

template <int TILE, bool NRM>
static int fwd_t(const HostPlan& P, const Batch* dB, float* image, float* alpha, float* depth,
                 float* normal, cudaStream_t st) {
  const int g = P.blend_fwd_blocks;
  // the backward's task list and overflow flag start empty for each forward
  if (P.px_clear && cudaMemsetAsync(P.px_clear, 0, 2 * sizeof(unsigned), st) != cudaSuccess)
    note_launch_error(cudaErrorInvalidValue);
  if (P.window > 0) {
    launch_k(k_blend_fwd_win<TILE, NRM>, dim3(g), dim3(WPB * 32), 0, st, dB, image, alpha, depth, normal);
    return 1;
  }
  switch (warps_index(P.blend_warps)) {
    case 0: fwd_nw<TILE, NRM, 2>(P, dB, image, alpha, depth, normal, st); break;
    case 2: fwd_nw<TILE, NRM, 8>(P, dB, image, alpha, depth, normal, st); break;
    default: fwd_nw<TILE, NRM, 4>(P, dB, image, alpha, depth, normal, st); break;
  }
  return 1;
}

template <int TILE, bool NRM, int NW>
static void bwd_nw(const HostPlan& P, const Batch* dB, const float* dimage, const float* dalpha,
                   const float* ddepth, const float* dnormal, const GradOut& zg, cudaStream_t st) {
  if (P.count)
    launch_k(k_blend_bwd<TILE, NRM, NW, true>, dim3(P.blend_bwd_blocks), dim3(NW * 32), 0, st, dB,
             dimage, dalpha, ddepth, dnormal, zg);
  else
    launch_k(k_blend_bwd<TILE, NRM, NW>, dim3(P.blend_bwd_blocks), dim3(NW * 32), 0, st, dB,
             dimage, dalpha, ddepth, dnormal, zg);
}

template <int TILE, bool NRM>
static int bwd_t(const HostPlan& P, const Batch* dB, const float* dimage, const float* dalpha,
                 const float* ddepth, const float* dnormal, const GradOut& zg, cudaStream_t st) {
  const int g = P.blend_bwd_blocks;
  int n = 1;
  if (P.frag_cap > 0 && P.window == 0) {
    launch_k(k_blend_bwd_px<TILE, NRM>, dim3(P.px_blocks), dim3(PXW * 32), 0, st, dB, dimage,
             dalpha, ddepth, dnormal, zg);
    n = 2;
  }
  if (P.window > 0) {
    launch_k(k_blend_bwd_win<TILE, NRM>, dim3(g), dim3(WPB * 32), 0, st, dB, dimage, dalpha, ddepth,
             dnormal, zg);
    return n;
  }
  switch (warps_index(P.blend_warps)) {
    case 0: bwd_nw<TILE, NRM, 2>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st); break;
    case 2: bwd_nw<TILE, NRM, 8>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st); break;
    default: bwd_nw<TILE, NRM, 4>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st); break;
  }
  return n;
}

int launch_blend_fwd(const HostPlan& P, const Batch* dB, float* image, float* alpha, float* depth,
                     float* normal, cudaStream_t st) {
  switch (P.tile * 2 + (P.normals ? 1 : 0)) {
    case 16: return fwd_t<8, false>(P, dB, image, alpha, depth, normal, st);
    case 17: return fwd_t<8, true>(P, dB, image, alpha, depth, normal, st);
    case 32: return fwd_t<16, false>(P, dB, image, alpha, depth, normal, st);
    case 33: return fwd_t<16, true>(P, dB, image, alpha, depth, normal, st);
    case 64: return fwd_t<32, false>(P, dB, image, alpha, depth, normal, st);
    default: return fwd_t<32, true>(P, dB, image, alpha, depth, normal, st);
  }
}

int launch_blend_bwd(const HostPlan& P, const Batch* dB, const float* dimage, const float* dalpha,
                     const float* ddepth, const float* dnormal, const GradOut* zero,
                     cudaStream_t st) {
  GradOut zg;
  if (zero) zg = *zero;
  else zg.dV[0] = nullptr;
  switch (P.tile * 2 + (P.normals ? 1 : 0)) {
    case 16: return bwd_t<8, false>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st);
    case 17: return bwd_t<8, true>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st);
    case 32: return bwd_t<16, false>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st);
    case 33: return bwd_t<16, true>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st);
    case 64: return bwd_t<32, false>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st);
    default: return bwd_t<32, true>(P, dB, dimage, dalpha, ddepth, dnormal, zg, st);
  }
}

int launch_zero_grads(const HostPlan& P, const Batch* dB, const GradOut& go, cudaStream_t st) {
  launch_k(k_zero_grads, dim3(P.tet_bwd_blocks * 4, P.n_scenes), dim3(256), 0, st, dB, go);
  return 1;
}

int launch_tet_bwd(const HostPlan& P, const Batch* dB, const GradOut& go, cudaStream_t st) {
  dim3 g(P.tet_bwd_blocks, P.n_scenes);
  if (P.normals) launch_k(k_tet_bwd<true>, dim3(g), dim3(TB_WARPS * 32), 0, st, dB, go);
  else launch_k(k_tet_bwd<false>, dim3(g), dim3(TB_WARPS * 32), 0, st, dB, go);
  return 1;
}

}  // namespace tts
