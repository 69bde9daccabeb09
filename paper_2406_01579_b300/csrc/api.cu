// C ABI of libtets: argument checks, workspace layout, launch sequences.
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <vector>

#include "launch.h"

namespace tts {

static_assert(sizeof(Batch) < 30000, "descriptor must fit in kernel parameters");

// Copies the by-value descriptor into the workspace (kernel parameters are
// captured by value in CUDA graphs, so this stays valid under capture): the
// header and the batch's scene and view entries only.
static_assert(offsetof(Batch, sc) % 4 == 0 && sizeof(SceneD) % 4 == 0 && sizeof(ViewD) % 4 == 0,
              "word copies");

__global__ void k_upload(const Batch b, Batch* dst) {
  pdl_wait();
  pdl_launch_dependents();
  const unsigned* src = reinterpret_cast<const unsigned*>(&b);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  constexpr int oS = (int)(offsetof(Batch, sc) / 4), oV = (int)(offsetof(Batch, vw) / 4),
                oSV = (int)(offsetof(Batch, scene_views) / 4);
  const int nS = b.n_scenes * (int)(sizeof(SceneD) / 4), nV = b.n_views * (int)(sizeof(ViewD) / 4);
  const int n = oS + nS + nV + b.n_views;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int w = (i < oS) ? i : (i < oS + nS) ? i : (i < oS + nS + nV) ? oV + (i - oS - nS)
                                                                        : oSV + (i - oS - nS - nV);
    d[w] = src[w];
  }
}

int launch_upload(const Batch& hb, Batch* dB, cudaStream_t st) {
  launch_k(k_upload, dim3(1), dim3(256), 0, st, hb, dB);
  return 1;
}

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_launch_err{0};

// Tile-scan look-back waits (tts_debug_scan_wait): polls before giving up,
// and the scan block made to poll a word that is never published (-1: none).
constexpr long long kScanSpinLimit = 1ll << 22;
static std::atomic<long long> g_scan_spin_limit{kScanSpinLimit};
static std::atomic<int> g_scan_unset_block{-1};

void count_launches(long long n) { g_launches += n; }
void note_launch_error(cudaError_t e) { g_launch_err.store((int)e); }

// Kernel-event hook (tts_debug_kernel_events): events recorded after each
// launch_k launch, with the kernels' names.  Off (n == 0) by default.
static std::atomic<int> g_kev_n{0}, g_kev_i{0};
static cudaEvent_t g_kev[256];
static const char* g_kev_name[256];

void note_kernel_launched(const void* kernel, cudaStream_t st) {
  if (g_kev_n.load(std::memory_order_relaxed) == 0) return;
  const int i = g_kev_i.fetch_add(1);
  if (i >= g_kev_n.load()) return;
  const char* name = nullptr;
  if (cudaFuncGetName(&name, kernel) != cudaSuccess) name = "?";
  g_kev_name[i] = name;
  if (cudaEventRecord(g_kev[i], st) != cudaSuccess) note_launch_error(cudaErrorInvalidValue);
}

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr int kBlendSegment = 256;    // default list entries per backward segment

int bit_length(long long x) {
  int b = 0;
  while (x > 0) { ++b; x >>= 1; }
  return b;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

struct Plan {
  Batch hb;      // descriptor with device pointers filled in
  HostPlan hp;
  size_t bytes;
  size_t off_desc;
  size_t off_ctr, off_rec_grad, bytes_rec_grad;
};

// Validates the batch and computes the workspace layout.  When base is null
// only sizes are computed.
int make_plan(const tts_batch* b, Plan* P, bool need_ws) {
  if (!b || !b->scenes || !b->views) return TTS_ERR_ARG;
  if (b->n_scenes < 1 || b->n_scenes > TTS_MAX_SCENES) return TTS_ERR_ARG;
  if (b->n_views < 1 || b->n_views > TTS_MAX_VIEWS) return TTS_ERR_ARG;
  const tts_params& pr = b->params;
  if (!(pr.tile == 8 || pr.tile == 16 || pr.tile == 32)) return TTS_ERR_ARG;
  if (!(std::isfinite(pr.s) && pr.s > 0.f)) return TTS_ERR_ARG;
  if (!(pr.alpha_cap > 0.f && pr.alpha_cap <= 1.f && pr.t_eps >= 0.f && pr.alpha_skip >= 0.f &&
        pr.prefilter_thresh >= 0.f))
    return TTS_ERR_ARG;
  if (b->key_capacity < 1 || b->key_capacity > 0x7fffffffLL) return TTS_ERR_ARG;
  if (pr.resort_window < 0 || pr.resort_window > 7) return TTS_ERR_ARG;
  if (pr.blend_segment != 0 &&
      (pr.blend_segment < 32 || pr.blend_segment > 65536 || pr.blend_segment % 32 != 0))
    return TTS_ERR_ARG;
  if (!(pr.blend_warps == 0 || pr.blend_warps == 2 || pr.blend_warps == 4 || pr.blend_warps == 8))
    return TTS_ERR_ARG;
  if (pr.frag_cap < -1 || pr.frag_cap > 255) return TTS_ERR_ARG;
  if (pr.flags & ~(TTS_FLAG_PURE | TTS_FLAG_ACCUM_GRAD | TTS_FLAG_FORWARD_ONLY | TTS_FLAG_NORMALS |
                   TTS_FLAG_HULL | TTS_FLAG_COUNT))
    return TTS_ERR_ARG;
  std::memset(&P->hb, 0, sizeof(Batch));
  Batch& B = P->hb;
  B.n_scenes = b->n_scenes;
  B.n_views = b->n_views;
  B.s = pr.s;
  B.prefilter_thresh = pr.prefilter_thresh;
  B.alpha_skip = pr.alpha_skip;
  B.alpha_cap = pr.alpha_cap;
  B.t_eps = pr.t_eps;
  B.tile = pr.tile;
  B.flags = pr.flags;
  B.resort_window = pr.resort_window;
  B.seg_len = (pr.resort_window > 0) ? 0 : (pr.blend_segment > 0 ? pr.blend_segment : kBlendSegment);
  B.key_cap = b->key_capacity;
  B.ts_spin_limit = g_scan_spin_limit.load();
  B.ts_unset_block = g_scan_unset_block.load();
  // scenes
  long long surv_total = 0, flag_total = 0, max_surv = 1;
  int pf_chunks = 0, max_pf = 1;
  std::vector<int> views_of(b->n_scenes, 0);
  for (int v = 0; v < b->n_views; ++v) {
    const int s = b->views[v].scene;
    if (s < 0 || s >= b->n_scenes) return TTS_ERR_ARG;
    views_of[s]++;
  }
  int voff = 0;
  for (int s = 0; s < b->n_scenes; ++s) {
    const tts_scene& sc = b->scenes[s];
    if (!sc.V || !sc.T || !sc.f || !sc.rgb) return TTS_ERR_ARG;
    if (sc.N < 1 || sc.K < 1 || sc.K > 0x7fffffffLL || sc.N > 0x7fffffffLL) return TTS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(sc.T) % 16 != 0) return TTS_ERR_ARG;  // int4 loads
    SceneD& S = B.sc[s];
    S.V = sc.V;
    S.T = reinterpret_cast<const int4*>(sc.T);
    S.f = sc.f;
    S.rgb = sc.rgb;
    S.N = sc.N;
    S.K = sc.K;
    S.surv_cap = (sc.surv_capacity > 0) ? std::min<long long>(sc.surv_capacity, sc.K) : sc.K;
    S.surv_off = surv_total;
    surv_total += S.surv_cap;
    max_surv = std::max(max_surv, S.surv_cap);
    S.flag_off = flag_total;
    flag_total += align_up(sc.K, 16);
    S.pf_chunks = (int)((sc.K + PF_CHUNK - 1) / PF_CHUNK);
    S.pf_chunk_base = pf_chunks;
    pf_chunks += S.pf_chunks;
    max_pf = std::max(max_pf, S.pf_chunks);
    S.view_off = voff;
    S.view_cnt = 0;
    voff += views_of[s];
  }
  // views
  long long slots = 0, pix = 0;
  int tiles = 0, max_pp = 1;
  for (int v = 0; v < b->n_views; ++v) {
    const tts_view& tv = b->views[v];
    const tts_camera& c = tv.cam;
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return TTS_ERR_ARG;
    if (!(c.fx > 0.f && c.fy > 0.f && std::isfinite(c.cx) && std::isfinite(c.cy) && c.znear > 0.f))
      return TTS_ERR_ARG;
    for (int i = 0; i < 9; ++i) if (!std::isfinite(c.R[i])) return TTS_ERR_ARG;
    for (int i = 0; i < 3; ++i) if (!std::isfinite(c.t[i])) return TTS_ERR_ARG;
    ViewD& V = B.vw[v];
    std::memcpy(V.R, c.R, sizeof(V.R));
    std::memcpy(V.t, c.t, sizeof(V.t));
    V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy; V.znear = c.znear;
    V.W = c.width; V.H = c.height;
    V.tiles_x = (c.width + pr.tile - 1) / pr.tile;
    V.tiles_y = (c.height + pr.tile - 1) / pr.tile;
    V.scene = tv.scene;
    V.tile_base = tiles;
    tiles += V.tiles_x * V.tiles_y;
    V.pix_base = pix;
    pix += (long long)c.width * c.height;
    V.rec_base = slots;
    const long long cap = B.sc[tv.scene].surv_cap;
    slots += cap;
    V.pp_chunks = (int)((cap + PP_CHUNK - 1) / PP_CHUNK);
    max_pp = std::max(max_pp, V.pp_chunks);
    SceneD& S = B.sc[tv.scene];
    B.scene_views[S.view_off + S.view_cnt++] = v;
  }
  if (slots > 0xffffffffLL) return TTS_ERR_ARG;  // 32-bit key values
  B.total_tiles = tiles;
  B.tile_bits = std::max(1, bit_length(tiles - 1));
  B.pf_chunks_total = pf_chunks;
  B.max_pf_chunks = max_pf;
  B.max_pp_chunks = max_pp;
  B.total_pixels = pix;
  B.total_slots = slots;
  // layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    const size_t r = off;
    off += bytes;
    return r;
  };
  const long long cap = b->key_capacity;
  P->off_desc = take(sizeof(Batch));
  P->off_ctr = take(sizeof(Counters));
  const size_t o_pfb = take(sizeof(int) * pf_chunks);
  const size_t o_pff = take((size_t)flag_total);
  const size_t o_bnd = take(sizeof(unsigned) * 6 * b->n_scenes);
  const size_t o_surv = take(sizeof(int) * surv_total);
  const size_t o_survT = take(sizeof(int4) * surv_total);
  const size_t o_rz = take(sizeof(unsigned) * slots);
  const size_t o_rr = take(sizeof(int4) * slots);
  const size_t o_rec = take(sizeof(float4) * REC_Q * slots);
  const bool fwd_only = (pr.flags & TTS_FLAG_FORWARD_ONLY) != 0;
  // record gradients and their touched flags, cleared together at init
  const size_t rg_bytes = sizeof(float4) * REC_Q * slots;
  P->bytes_rec_grad = fwd_only ? 0 : rg_bytes + (((size_t)slots + 15) & ~(size_t)15);
  P->off_rec_grad = take(P->bytes_rec_grad);
  const size_t o_k0 = take(sizeof(unsigned long long) * cap);
  const size_t o_k1 = take(sizeof(unsigned long long) * cap);
  const size_t o_v = take(sizeof(unsigned) * cap);
  const size_t o_tc = take(sizeof(int) * tiles);
  const size_t o_tcl = take(sizeof(int) * TSORT_CLASSES * (size_t)tiles);
  const size_t o_slb = take(sizeof(unsigned long long) * (size_t)((tiles + TS_TILES - 1) / TS_TILES));
  const size_t o_rng = take(sizeof(int2) * tiles);
  // split-tile segments: at most 2 * keys / seg_len (each split tile has more
  // than seg_len keys, so ceil(len / seg_len) <= 2 len / seg_len); one
  // checkpoint of 32 B per pixel and segment
  B.seg_cap = B.seg_len > 0 ? (int)std::min<long long>(2 * cap / B.seg_len + 1, 0x3fffffffLL) : 0;
  const long long tt = (long long)pr.tile * pr.tile;
  // forward units: one per tile, four per split tile; backward units: one
  // per tile, one per segment of a split tile
  const size_t o_wl = take(sizeof(int2) * 4 * (size_t)tiles);
  const size_t o_wlbk = take(sizeof(int2) * ((size_t)tiles + (size_t)B.seg_cap));
  const size_t o_tseg = take(sizeof(int2) * tiles);
  const size_t o_tlast = take(sizeof(int) * tiles);
  const int wl_blocks = (tiles + 255) / 256;
  const size_t o_wlc = take(sizeof(int) * 68 * (size_t)wl_blocks);
  const size_t o_wlb = take(sizeof(int) * 68);
  const size_t o_psa = take(sizeof(float4) * B.seg_cap * tt);
  const size_t o_psb = take(sizeof(float4) * B.seg_cap * tt);

  const size_t o_pT = take(sizeof(float) * pix);
  const size_t o_pL = take(sizeof(int) * pix);
  const size_t o_pN = take(sizeof(int) * pix);
  const size_t o_pC = take(sizeof(float4) * pix);
  const bool normals = (pr.flags & TTS_FLAG_NORMALS) != 0;
  const size_t o_sn = take(normals ? sizeof(float4) * surv_total : 0);
  const size_t o_pNm = take((normals && !fwd_only) ? sizeof(float4) * pix : 0);
  // per-pixel fragment lists (slot of each blended fragment, planar by index),
  // their lengths and the tiles holding a pixel past the cap
  const int fcap = (fwd_only || pr.resort_window > 0 || pr.frag_cap < 0 || pix > 0xffffffffLL)
                       ? 0
                       : (pr.frag_cap == 0 ? kFragCapDefault : pr.frag_cap);
  B.frag_cap = fcap;
  const size_t o_frag = take(fcap > 0 ? sizeof(unsigned) * (size_t)fcap * pix : 0);
  const size_t o_pnb = take(fcap > 0 ? sizeof(int) * pix : 0);
  const size_t o_tovf = take(fcap > 0 ? sizeof(int) * tiles : 0);
  const size_t o_pxl = take(fcap > 0 ? sizeof(uint2) * pix : 0);
  P->bytes = align_up(off, 256);
  if (need_ws) {
    if (!b->workspace || (reinterpret_cast<uintptr_t>(b->workspace) % 256) != 0)
      return TTS_ERR_WORKSPACE;
    if (b->workspace_bytes < P->bytes) return TTS_ERR_WORKSPACE;
    char* base = static_cast<char*>(b->workspace);
    B.ctr = reinterpret_cast<Counters*>(base + P->off_ctr);
    B.pf_blocksum = reinterpret_cast<int*>(base + o_pfb);
    B.pf_flags = reinterpret_cast<unsigned char*>(base + o_pff);
    B.bounds = reinterpret_cast<unsigned*>(base + o_bnd);
    B.surv = reinterpret_cast<int*>(base + o_surv);
    B.surv_T = reinterpret_cast<int4*>(base + o_survT);
    B.rec_z = reinterpret_cast<unsigned*>(base + o_rz);
    B.rec_rect = reinterpret_cast<int4*>(base + o_rr);
    B.rec = reinterpret_cast<float4*>(base + o_rec);
    B.rec_grad = reinterpret_cast<float4*>(base + P->off_rec_grad);
    B.rec_touched = fwd_only ? nullptr : reinterpret_cast<unsigned char*>(base + P->off_rec_grad + rg_bytes);
    B.keys[0] = reinterpret_cast<unsigned long long*>(base + o_k0);
    B.keys[1] = reinterpret_cast<unsigned long long*>(base + o_k1);
    B.vals = reinterpret_cast<unsigned*>(base + o_v);
    B.tile_cnt = reinterpret_cast<int*>(base + o_tc);
    B.tile_class = reinterpret_cast<int*>(base + o_tcl);
    B.scan_lb = reinterpret_cast<unsigned long long*>(base + o_slb);
    B.ranges = reinterpret_cast<int2*>(base + o_rng);
    B.worklist = reinterpret_cast<int2*>(base + o_wl);
    B.worklist_b = reinterpret_cast<int2*>(base + o_wlbk);
    B.tseg = reinterpret_cast<int2*>(base + o_tseg);
    B.tile_last = reinterpret_cast<int*>(base + o_tlast);
    B.wl_blockcnt = reinterpret_cast<int*>(base + o_wlc);
    B.wl_base = reinterpret_cast<int*>(base + o_wlb);
    B.pseg_a = reinterpret_cast<float4*>(base + o_psa);
    B.pseg_b = reinterpret_cast<float4*>(base + o_psb);

    B.pix_T = reinterpret_cast<float*>(base + o_pT);
    B.pix_last = reinterpret_cast<int*>(base + o_pL);
    B.pix_nfrag = reinterpret_cast<int*>(base + o_pN);
    B.pix_CD = reinterpret_cast<float4*>(base + o_pC);
    B.surv_n = normals ? reinterpret_cast<float4*>(base + o_sn) : nullptr;
    B.pix_N = (normals && !fwd_only) ? reinterpret_cast<float4*>(base + o_pNm) : nullptr;
    B.frag = fcap > 0 ? reinterpret_cast<unsigned*>(base + o_frag) : nullptr;
    B.pix_nb = fcap > 0 ? reinterpret_cast<int*>(base + o_pnb) : nullptr;
    B.tile_ovf = fcap > 0 ? reinterpret_cast<int*>(base + o_tovf) : nullptr;
    B.px_list = fcap > 0 ? reinterpret_cast<uint2*>(base + o_pxl) : nullptr;
  }
  HostPlan& H = P->hp;
  H.n_scenes = b->n_scenes;
  H.n_views = b->n_views;
  H.max_pf_chunks = max_pf;
  H.max_pp_chunks = max_pp;
  H.max_pre_chunks = (int)((max_surv + PRE_CHUNK - 1) / PRE_CHUNK);
  H.tsort_blocks = std::max(1, std::min(tiles, TSORT_BLOCKS_PER_SM * sm_count()));
  H.wl_blocks = wl_blocks;
  H.total_tiles = tiles;
  H.tile = pr.tile;
  H.window = pr.resort_window;
  H.normals = normals;
  H.hull = (pr.flags & TTS_FLAG_HULL) != 0;
  H.count = (pr.flags & TTS_FLAG_COUNT) != 0;
  H.normal_blocks = (int)std::min<long long>((max_surv + 255) / 256, 8LL * sm_count());
  H.tet_bwd_blocks = 4 * sm_count();
  H.blend_warps = pr.blend_warps > 0 ? pr.blend_warps : 4;
  H.frag_cap = fcap;
  H.px_clear = (need_ws && fcap > 0) ? &B.ctr->px_n : nullptr;
  H.px_blocks = fcap > 0 ? px_grid(pr.tile, normals, sm_count()) : 0;
  blend_grid(pr.tile, normals, pr.resort_window, H.blend_warps, sm_count(), &H.blend_fwd_blocks,
             &H.blend_bwd_blocks);
  H.total_pixels = pix;
  return TTS_OK;
}

Batch* dev_desc(const tts_batch* b, const Plan& P) {
  return reinterpret_cast<Batch*>(static_cast<char*>(b->workspace) + P.off_desc);
}

int check_launch() {
  const cudaError_t e = cudaPeekAtLastError();
  const int le = g_launch_err.exchange(0);
  return (e == cudaSuccess && le == 0) ? TTS_OK : TTS_ERR_CUDA;
}

}  // namespace
}  // namespace tts

using namespace tts;

extern "C" {

int tts_workspace_size(const tts_batch* b, size_t* bytes) {
  if (!bytes) return TTS_ERR_ARG;
  Plan P;
  const int rc = make_plan(b, &P, false);
  if (rc != TTS_OK) return rc;
  *bytes = P.bytes;
  return TTS_OK;
}

int tts_workspace_init(const tts_batch* b, tts_stream stream) {
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(b->workspace);
  if (cudaMemsetAsync(base + P.off_ctr, 0, sizeof(Counters), st) != cudaSuccess) return TTS_ERR_CUDA;
  if (P.bytes_rec_grad &&
      cudaMemsetAsync(base + P.off_rec_grad, 0, P.bytes_rec_grad, st) != cudaSuccess)
    return TTS_ERR_CUDA;

  return TTS_OK;
}

int tts_prepare_scene(const tts_batch* b, tts_stream stream) {
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Batch* dB = dev_desc(b, P);
  long long n = launch_upload(P.hb, dB, st);
  n += launch_prefilter(P.hp, dB, st);
  g_launches += n;
  return check_launch();
}

int tts_survivor_bounds(const tts_batch* b, float* aabb, tts_stream stream) {
  if (!aabb) return TTS_ERR_ARG;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  g_launches += launch_bounds(P.hp, dev_desc(b, P), aabb, st);
  return check_launch();
}

int tts_fit_grid(const float* V_in, int64_t N, const float grid_lo[3], const float grid_hi[3],
                 const float* aabb, float pad, float* V_out, tts_stream stream) {
  if (!V_in || !V_out || !aabb || !grid_lo || !grid_hi || N < 1 || N > 0x7fffffffLL) return TTS_ERR_ARG;
  if (!(std::isfinite(pad) && pad >= 0.f)) return TTS_ERR_ARG;
  float lo[3], hi[3];
  for (int i = 0; i < 3; ++i) {
    lo[i] = grid_lo[i];
    hi[i] = grid_hi[i];
    if (!(std::isfinite(lo[i]) && std::isfinite(hi[i]) && hi[i] > lo[i])) return TTS_ERR_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  g_launches += launch_fit_grid(V_in, N, lo, hi, aabb, pad, V_out, st);
  return check_launch();
}

int tts_bin_views(const tts_batch* b, tts_stream stream) {
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Batch* dB = dev_desc(b, P);
  long long n = launch_upload(P.hb, dB, st);
  n += launch_binning(P.hp, dB, st);
  g_launches += n;
  return check_launch();
}

static bool outputs_ok(const tts_batch* b, const tts_outputs* o) {
  if (!b || !o || !o->image || !o->alpha || !o->depth) return false;
  const bool normals = (b->params.flags & TTS_FLAG_NORMALS) != 0;
  return normals == (o->normal != nullptr);
}

static bool upstream_ok(const tts_batch* b, const tts_upstream* u) {
  if (!b || !u || !u->dimage || (b->params.flags & TTS_FLAG_FORWARD_ONLY)) return false;
  return u->dnormal == nullptr || (b->params.flags & TTS_FLAG_NORMALS) != 0;
}

int tts_blend_fwd_ex(const tts_batch* b, const tts_outputs* out, tts_stream stream) {
  if (!outputs_ok(b, out)) return TTS_ERR_ARG;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  g_launches += launch_blend_fwd(P.hp, dev_desc(b, P), out->image, out->alpha, out->depth,
                                 out->normal, st);
  return check_launch();
}

int tts_blend_fwd(const tts_batch* b, float* image, float* alpha, float* depth, tts_stream stream) {
  const tts_outputs o = {image, alpha, depth, nullptr};
  return tts_blend_fwd_ex(b, &o, stream);
}

int tts_render_fwd_ex(const tts_batch* b, const tts_outputs* out, tts_stream stream) {
  if (!outputs_ok(b, out)) return TTS_ERR_ARG;
  int rc = tts_bin_views(b, stream);
  if (rc != TTS_OK) return rc;
  return tts_blend_fwd_ex(b, out, stream);
}

int tts_render_fwd(const tts_batch* b, float* image, float* alpha, float* depth, tts_stream stream) {
  const tts_outputs o = {image, alpha, depth, nullptr};
  return tts_render_fwd_ex(b, &o, stream);
}

// The blend backward; with zero, its warps also clear those vertex-gradient
// arrays once their work is done (for a record -> vertex scatter that
// follows without clearing).
static int blend_bwd_impl(const tts_batch* b, const tts_upstream* up, const GradOut* zero,
                          tts_stream stream) {
  if (!upstream_ok(b, up)) return TTS_ERR_ARG;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  g_launches += launch_blend_bwd(P.hp, dev_desc(b, P), up->dimage, up->dalpha, up->ddepth,
                                 up->dnormal, zero, st);
  return check_launch();
}

int tts_blend_bwd_ex(const tts_batch* b, const tts_upstream* up, tts_stream stream) {
  return blend_bwd_impl(b, up, nullptr, stream);
}

int tts_blend_bwd(const tts_batch* b, const float* dimage, const float* dalpha, const float* ddepth,
                  tts_stream stream) {
  const tts_upstream u = {dimage, dalpha, ddepth, nullptr};
  return tts_blend_bwd_ex(b, &u, stream);
}

static int grad_out(const tts_batch* b, float* const* dV, float* const* df, float* const* drgb,
                    GradOut* go) {
  if (!dV || !df || !drgb || !b || (b->params.flags & TTS_FLAG_FORWARD_ONLY)) return TTS_ERR_ARG;
  if (b->n_scenes < 1 || b->n_scenes > TTS_MAX_SCENES) return TTS_ERR_ARG;
  std::memset(go, 0, sizeof(*go));
  for (int s = 0; s < b->n_scenes; ++s) {
    if (!dV[s] || !df[s] || !drgb[s]) return TTS_ERR_ARG;
    go->dV[s] = dV[s];
    go->df[s] = df[s];
    go->drgb[s] = drgb[s];
  }
  return TTS_OK;
}

// The record -> vertex scatter; `cleared`: the gradient arrays were already
// cleared (by the blend backward) and must not be cleared again.
static int scatter_bwd_impl(const tts_batch* b, const GradOut& go, bool cleared, tts_stream stream) {
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!cleared && !(b->params.flags & TTS_FLAG_ACCUM_GRAD))
    g_launches += launch_zero_grads(P.hp, dev_desc(b, P), go, st);
  g_launches += launch_tet_bwd(P.hp, dev_desc(b, P), go, st);
  return check_launch();
}

int tts_scatter_bwd(const tts_batch* b, float* const* dV, float* const* df, float* const* drgb,
                    tts_stream stream) {
  GradOut go;
  int rc = grad_out(b, dV, df, drgb, &go);
  if (rc != TTS_OK) return rc;
  return scatter_bwd_impl(b, go, false, stream);
}

int tts_render_bwd_ex(const tts_batch* b, const tts_upstream* up, float* const* dV,
                      float* const* df, float* const* drgb, tts_stream stream) {
  if (!upstream_ok(b, up)) return TTS_ERR_ARG;
  GradOut go;
  int rc = grad_out(b, dV, df, drgb, &go);
  if (rc != TTS_OK) return rc;
  // the blend backward clears the gradients as its warps run out of work
  const bool clear = !(b->params.flags & TTS_FLAG_ACCUM_GRAD);
  rc = blend_bwd_impl(b, up, clear ? &go : nullptr, stream);
  if (rc != TTS_OK) return rc;
  return scatter_bwd_impl(b, go, clear, stream);
}

int tts_render_bwd(const tts_batch* b, const float* dimage, const float* dalpha, const float* ddepth,
                   float* const* dV, float* const* df, float* const* drgb, tts_stream stream) {
  const tts_upstream u = {dimage, dalpha, ddepth, nullptr};
  return tts_render_bwd_ex(b, &u, dV, df, drgb, stream);
}

int64_t tts_launch_count(void) { return g_launches.load(); }

int tts_debug_kernel_events(void* const* events, int32_t n) {
  if (n < 0 || n > 256 || (n > 0 && !events)) return TTS_ERR_ARG;
  g_kev_n.store(0);
  for (int i = 0; i < n; ++i) g_kev[i] = static_cast<cudaEvent_t>(events[i]);
  g_kev_i.store(0);
  g_kev_n.store(n);
  return TTS_OK;
}

int32_t tts_debug_kernel_events_used(const char** names, int32_t max_names) {
  const int used = std::min(g_kev_i.load(), g_kev_n.load());
  for (int i = 0; names && i < std::min(used, (int)max_names); ++i) names[i] = g_kev_name[i];
  return used;
}

int tts_debug_scan_wait(int64_t spin_limit, int32_t unset_block) {
  if (spin_limit < 0 || unset_block < -1) return TTS_ERR_ARG;
  g_scan_spin_limit.store(spin_limit == 0 ? kScanSpinLimit : spin_limit);
  g_scan_unset_block.store(unset_block);
  return TTS_OK;
}

int tts_debug_pixels(const tts_batch* b, const void** T_final, const void** last,
                     const void** n_frag, tts_stream stream) {
  (void)stream;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  if (T_final) *T_final = P.hb.pix_T;
  if (last) *last = P.hb.pix_last;
  if (n_frag) *n_frag = P.hb.pix_nfrag;
  return TTS_OK;
}

int tts_debug_walk_counts(const tts_batch* b, uint64_t counts[5], int32_t reset,
                          tts_stream stream) {
  if (!counts) return TTS_ERR_ARG;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* w = P.hb.ctr->walk;
  if (cudaMemcpyAsync(counts, w, 5 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TTS_ERR_CUDA;
  if (reset && cudaMemsetAsync(w, 0, 5 * sizeof(uint64_t), st) != cudaSuccess) return TTS_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? TTS_OK : TTS_ERR_CUDA;
}

int tts_debug_frag_lists(const tts_batch* b, const void** frag, const void** n_blend,
                         const void** tile_over, int32_t* frag_cap, tts_stream stream) {
  (void)stream;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  if (frag) *frag = P.hb.frag;
  if (n_blend) *n_blend = P.hb.pix_nb;
  if (tile_over) *tile_over = P.hb.tile_ovf;
  if (frag_cap) *frag_cap = P.hb.frag_cap;
  return TTS_OK;
}

int tts_get_info(const tts_batch* b, tts_info* info, tts_stream stream) {
  if (!info) return TTS_ERR_ARG;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Counters c;
  if (cudaMemcpyAsync(&c, P.hb.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TTS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TTS_ERR_CUDA;
  std::memset(info, 0, sizeof(*info));
  info->status = c.status;
  info->n_scenes = b->n_scenes;
  info->n_keys = c.n_keys;
  for (int s = 0; s < b->n_scenes; ++s) info->n_surv[s] = c.n_surv[s];
  info->sort_bits = c.total_bits;
  info->long_lists = c.long_lists;
  info->blend_units = c.n_units_b;
  return TTS_OK;
}

int tts_debug_lists(const tts_batch* b, const void** keys, const void** vals, const void** ranges,
                    const void** surv, uint32_t* zmin_bits, int32_t* depth_bits, tts_stream stream) {
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (keys) {
    g_launches += launch_debug_keys(P.hp, dev_desc(b, P), st);
    if (check_launch() != TTS_OK) return TTS_ERR_CUDA;
  }
  Counters c;
  if (cudaMemcpyAsync(&c, P.hb.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TTS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TTS_ERR_CUDA;
  if (keys) *keys = P.hb.keys[0];
  if (vals) *vals = P.hb.vals;
  if (ranges) *ranges = P.hb.ranges;
  if (surv) *surv = P.hb.surv;
  if (zmin_bits) *zmin_bits = c.zmin_bits;
  if (depth_bits) *depth_bits = c.depth_bits;
  return TTS_OK;
}

int tts_debug_records(const tts_batch* b, const void** records, tts_stream stream) {
  (void)stream;
  Plan P;
  int rc = make_plan(b, &P, true);
  if (rc != TTS_OK) return rc;
  if (records) *records = P.hb.rec;
  return TTS_OK;
}

const char* tts_error_string(int code) {
  switch (code) {
    case TTS_OK: return "ok";
    case TTS_ERR_ARG: return "invalid argument";
    case TTS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case TTS_ERR_OVERFLOW: return "key or survivor capacity exceeded";
    case TTS_ERR_CUDA: return "CUDA error";
    case TTS_ERR_TIMEOUT: return "device wait timed out";
    case TTS_ERR_BAD_INDEX: return "tet index outside [0, N)";
    default: return "unknown error";
  }
}

const char* tts_version(void) { return "libtets 0.1 sm_103a"; }

}  // extern "C"
