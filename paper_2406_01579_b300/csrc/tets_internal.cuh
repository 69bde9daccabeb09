// Internal device-side definitions of libtets: the batch descriptor, the
// workspace counters, the per-(view, tet) record and the chord/opacity
// evaluation shared by the forward and backward blend kernels.
#pragma once

#include <cstddef>

#include <cstdint>
#include <cuda_runtime.h>

#include "tets.h"

namespace tts {

constexpr int PF_CHUNK = 2048;      // tets per pre-filter block (32 KB of indices in shared memory)
constexpr int PF_THREADS = 256;
constexpr int PP_CHUNK = 512;       // slots per key placement block
constexpr int PRE_THREADS = 128;    // preprocess block
constexpr int PRE_CHUNK = 128;      // survivors per preprocess block
constexpr int PP_THREADS = 256;
constexpr int SCAN_THREADS = 1024;
constexpr int TS_THREADS = 256;     // tile scan: threads per block
constexpr int TS_ITEMS = 8;         // tiles per thread
constexpr int TS_TILES = TS_THREADS * TS_ITEMS;
constexpr int kFragCapDefault = 128;  // per-pixel fragment list capacity (tts_params.frag_cap 0)
constexpr int TSORT_BLOCKS_PER_SM = 4;   // resident blocks of the persistent depth sort
constexpr int TSORT_CLASSES = 6;    // depth-sort list lengths (0,256] (256,512] (512,1K] (1K,2K] (2K,4K] (4K,...)

// Counters at the start of the workspace (after the descriptor).
struct Counters {
  unsigned int status;
  unsigned int zmin_bits;   // min over all views of the FP32 mean depth bits
  unsigned int zmax_bits;
  int depth_bits;           // bits of (zbits - zmin_bits)
  int total_bits;           // depth_bits + tile_bits
  int long_lists;           // tiles sorted by the global-memory merge
  long long n_keys;         // keys produced (may exceed capacity: then overflow)
  long long n_keys_used;    // keys the sort and blend see (0 on overflow)
  int n_surv[TTS_MAX_SCENES];
  unsigned int work_fwd, work_bwd;      // persistent blend work queues
  unsigned int done_fwd, done_bwd;      // warps finished (last one resets)
  int n_units;              // forward work units (tile lists, 4x2-block parts) of the last binning
  int n_units_b;            // backward work units (tile lists and list segments)
  int seg_total;            // checkpoint slots handed out by the work-list builder
  int class_n[TSORT_CLASSES];   // tiles in each list-length class of the depth sort
  int sort_q[5];            // depth-sort queues: block, half, quarter, eighth and warp lists taken
  unsigned int scan_ticket; // tile-scan blocks started
  unsigned int zero_q;      // gradient-clearing chunks taken by the backward
  unsigned long long scan_unset; // a look-back word no kernel writes (the scan-wait test hook)
  unsigned int px_n;        // pixels in Batch::px_list (cleared before each forward)
  unsigned int ovf_any;     // 1: a pixel has more blended fragments than frag_cap (cleared with px_n)
  unsigned long long walk[5];   // TTS_FLAG_COUNT: walk statistics (tts_debug_walk_counts)
};
static_assert(offsetof(Counters, ovf_any) == offsetof(Counters, px_n) + 4,
              "px_n and ovf_any are cleared together");

struct SceneD {
  const float* V;
  const int4* T;
  const float* f;
  const float* rgb;
  long long N, K;
  long long surv_off;       // into the survivor buffer
  long long surv_cap;
  long long flag_off;       // into the pre-filter flag buffer
  int pf_chunk_base;        // first pre-filter block-sum slot
  int pf_chunks;
  int view_off, view_cnt;   // this scene's views in Batch::scene_views
};

struct ViewD {
  float R[9];
  float t[3];
  float fx, fy, cx, cy, znear;
  int W, H, tiles_x, tiles_y;
  int scene;
  int tile_base;            // first global tile id
  long long pix_base;       // first output pixel
  long long rec_base;       // first record slot
  int pp_chunks;            // preprocess / key placement blocks
};

struct Batch {
  int n_scenes, n_views;
  int total_tiles, tile_bits;
  int pf_chunks_total;
  int max_pf_chunks, max_pp_chunks;
  float s, prefilter_thresh, alpha_skip, alpha_cap, t_eps;
  int tile, flags;
  int resort_window;
  int seg_len;              // list entries per blend work unit (0: no splitting)
  int seg_cap;              // segment slots of the split-tile checkpoints
  int ts_unset_block;       // tile-scan block whose look-back reads Counters::scan_unset (-1: none)
  long long ts_spin_limit;  // polls of a tile-scan look-back word before it gives up
  long long key_cap;
  long long total_pixels;
  long long total_slots;
  // workspace regions
  Counters* ctr;
  int* pf_blocksum;         // [pf_chunks_total]
  unsigned char* pf_flags;  // [sum K]
  unsigned int* bounds;     // [6 * n_scenes] survivor AABB as order-preserving float keys
  int* surv;                // [sum surv_cap]
  int4* surv_T;             // [sum surv_cap] vertex ids of each survivor
  unsigned int* rec_z;      // [slots] FP32 mean depth bits
  int4* rec_rect;           // [slots] tile rect (tx0, tx1, ty0, ty1)
  float4* rec;              // [slots * 6]
  float4* rec_grad;         // [slots * 6] record gradient (self-clearing)
  unsigned char* rec_touched;    // [slots] 1 once the slot's gradient was added to (self-clearing)
  unsigned long long* keys[2];   // [key_cap] each: [1] (zbits << 32 | slot) bucketed by
                                 // tile; [0] merge scratch, debug keys on request
  unsigned int* vals;       // [key_cap] record slot of each key, sorted per tile
  int* tile_cnt;            // [total_tiles] keys per tile, then the placement cursor
  int* tile_class;          // [TSORT_CLASSES * total_tiles] non-empty tiles by list length
  unsigned long long* scan_lb;   // [tile-scan blocks] look-back words (flag << 62 | sum)
  int2* ranges;             // [total_tiles]
  int2* worklist;           // [forward units] (tile, part << 24), longest first
  int2* worklist_b;         // [backward units] (tile, segment), longest first
  int2* tseg;               // [total_tiles] (first segment slot or -1, segment count)
  int* tile_last;           // [total_tiles] largest blended entry + 1 of a split list's pixels
  int* wl_blockcnt;         // [work-list blocks * 68] units per list, length bucket and block
  int* wl_base;             // [68] first unit of each list's length buckets
  float4* pseg_a;           // [seg_cap * tile^2] forward state at each segment end: (T, C0, C1, C2)
  float4* pseg_b;           // [seg_cap * tile^2] (D, N0, N1, N2)
  float* pix_T;             // [total_pixels]
  int* pix_last;            // [total_pixels]
  int* pix_nfrag;           // [total_pixels]
  float4* pix_CD;           // [total_pixels] final (C0, C1, C2, D)
  float4* surv_n;           // [sum surv_cap] world unit normal per survivor (normals only)
  float4* pix_N;            // [total_pixels] final normal (normals with a backward)
  int frag_cap;             // per-pixel fragment list capacity (0: no lists)
  unsigned* frag;           // [frag_cap * total_pixels] slot of the i-th blended fragment of
                            // pixel p at frag[i * total_pixels + p]
  int* pix_nb;              // [total_pixels] blended fragments of the pixel (may exceed the cap)
  int* tile_ovf;            // [total_tiles] 1: a pixel of the tile has more than frag_cap
  uint2* px_list;           // [total_pixels] pixels with 1..frag_cap blended fragments:
                            // (pixel, blended count | view << 8)
  SceneD sc[TTS_MAX_SCENES];
  ViewD vw[TTS_MAX_VIEWS];
  int scene_views[TTS_MAX_VIEWS];
};

// ---------------------------------------------------------------------------
// Record: 6 float4 per (view, survivor) slot.
//   q0  bbox (+-(i0+.5), +-(j0+.5), i1+.5, j1+.5) in pixel-centre units; the
//       sign of .x / .y says whether face slot 1 / 2 is a front face
//       (negative: front).  Slot 0 is always front, slot 3 always back.
//   q1  P_k, q2  A_k, q3  B_k  for face slots k = 0..3.  With the pixel offset
//       (dx, dy) from the bbox corner pixel centre (i0+.5, j0+.5),
//       rho_k = 1 + P_k + A_k dx + B_k dy = z_r / t_k where t_k is the depth at
//       which the pixel ray meets face k's plane and z_r a per-tet reference
//       depth.  Entry: min rho over front faces; exit: max rho over back faces.
//   q4  (F, K0, Kx, Ky) = (s f(x_r), s g.x_r, s z_r g_x / fx, s z_r g_y / fy)
//       for the tet's affine SDF f(x) with gradient g and the reference point
//       x_r = z_r * ray(i0+.5, j0+.5).  Along the pixel ray, with
//       lin = Kx dx + Ky dy:  s f(t) = (F + lin) + (K0 + lin) (t - z_r) / z_r.
//   q5  (zbar, r, g, b): mean vertex depth (Eq. 2 depth) and mean colour.
// The record gradient buffer has the same layout; its q0.xyz holds dL/dn of
// the tet's world unit normal (normal map channel).
// ---------------------------------------------------------------------------
constexpr int REC_Q = 6;

struct Chord {
  bool hit;
  int kin, kout;      // face slots binding the entry and the exit
  float p_in, p_out;  // rho - 1 at entry and exit
  float dx, dy;
};

// Everything below uses explicitly rounded intrinsics so that the forward
// and the backward (which recomputes each fragment) agree bit for bit.
__device__ __forceinline__ Chord chord_eval(const float4& q0, const float4& q1,
                                            const float4& q2, const float4& q3,
                                            float px, float py) {
  Chord c;
  c.dx = __fsub_rn(px, fabsf(q0.x));
  c.dy = __fsub_rn(py, fabsf(q0.y));
  const float p0 = __fmaf_rn(q2.x, c.dx, __fmaf_rn(q3.x, c.dy, q1.x));
  const float p1 = __fmaf_rn(q2.y, c.dx, __fmaf_rn(q3.y, c.dy, q1.y));
  const float p2 = __fmaf_rn(q2.z, c.dx, __fmaf_rn(q3.z, c.dy, q1.z));
  const float p3 = __fmaf_rn(q2.w, c.dx, __fmaf_rn(q3.w, c.dy, q1.w));
  float pin = p0, pout = p3;
  int kin = 0, kout = 3;
  if (q0.x < 0.f) {
    if (p1 < pin) { pin = p1; kin = 1; }
  } else {
    if (p1 > pout) { pout = p1; kout = 1; }
  }
  if (q0.y < 0.f) {
    if (p2 < pin) { pin = p2; kin = 2; }
  } else {
    if (p2 > pout) { pout = p2; kout = 2; }
  }
  const bool inside = (c.dx >= 0.f) & (c.dy >= 0.f) & (px <= q0.z) & (py <= q0.w);
  c.hit = inside & (pin > pout) & (pout > -1.f);
  c.p_in = pin;
  c.p_out = pout;
  c.kin = kin;
  c.kout = kout;
  return c;
}

struct Opacity {
  float alpha;
  float x, y;         // s (f_prev - f_next) and s f_next
  float e1, B;        // exp(-x) and sigmoid(-y)
  float r, rho_in, rho_out, sGz;
};

// Hardware reciprocal (MUFU, about 1 ulp).  Deterministic, so the forward
// and the backward, which both evaluate the opacity through opacity_eval,
// agree bit for bit.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Eq. 1 in the rewrite -expm1(-s (f_prev - f_next)) * sigmoid(-s f_next),
// 0 unless f_prev > f_next.  The chord geometry (App. A.2's depths) enters
// through rho_in, rho_out: t_in = z_r / rho_in, t_out = z_r / rho_out.
// Branch free: e1 and B are evaluated for every chord (x and y clamped so the
// exponentials stay finite) and alpha is selected; the backward reads e1 and
// B only where alpha > 0.
__device__ __forceinline__ Opacity opacity_eval(const float4& q4, const Chord& c) {
  Opacity o;
  o.rho_in = __fadd_rn(1.f, c.p_in);
  o.rho_out = __fadd_rn(1.f, c.p_out);
  o.r = rcp_approx(__fmul_rn(o.rho_in, o.rho_out));
  const float lin = __fmaf_rn(q4.z, c.dx, __fmul_rn(q4.w, c.dy));
  const float sF0 = __fadd_rn(q4.x, lin);
  o.sGz = __fadd_rn(q4.y, lin);
  // x = s (f_prev - f_next) = sGz (p_out - p_in) / (rho_in rho_out)
  o.x = __fmul_rn(__fmul_rn(o.sGz, __fsub_rn(c.p_out, c.p_in)), o.r);
  // y = s f_next = sF0 - sGz p_out / rho_out
  o.y = __fmaf_rn(-__fmul_rn(o.sGz, c.p_out), __fmul_rn(o.rho_in, o.r), sF0);
  o.e1 = __expf(-fminf(fmaxf(o.x, 0.f), 80.f));
  const float e2 = __expf(fminf(o.y, 80.f));
  o.B = rcp_approx(__fadd_rn(1.f, e2));
  o.alpha = (o.x > 0.f) ? __fmul_rn(__fsub_rn(1.f, o.e1), o.B) : 0.f;
  return o;
}

// Programmatic dependent launch: a kernel of the step may be scheduled while
// its predecessor in the stream finishes.  pdl_wait, its first statement,
// blocks until the predecessor grid has completed and its writes are
// visible; pdl_launch_dependents lets the successor be scheduled once every
// block of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Lanes per pixel of the forward walk of a tile list split into nseg
// backward segments: 1 (8x4 blocks) for an unsplit list, 4 (4x2 blocks) for a
// split one.  The forward work list holds as many units (parts, TILE^2 / 32
// blocks each) for the list as it has lanes per pixel.
__device__ __forceinline__ int fwd_lanes(int nseg) { return (nseg <= 1) ? 1 : 4; }

__device__ __forceinline__ void set_status(Counters* c, unsigned int bit) {
  atomicOr(&c->status, bit);
}

// ---------------------------------------------------------------------------
// host-side launch wrappers (one per kernel group)
// ---------------------------------------------------------------------------
struct HostBatch;  // host mirror, defined in tets_api.cu

}  // namespace tts
