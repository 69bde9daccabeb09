/*
 * tets.h — C ABI of the tetrahedron splatting rasterizer (libtets.so).
 *
 * Renders structured or unstructured tetrahedral grids whose vertices carry a
 * signed distance value f and a colour, following "Tetrahedron Splatting for
 * 3D Generation" (TeT-Splatting), Sec. 3.2-3.3 and App. A:
 *
 *   tts_prepare_scene   pre-filter (Sec. 3.2 "Pre-filtering"): per tet
 *                       alpha_max = Eq. 1 at (max f, min f); keep the tets with
 *                       alpha_max >= T_f, in their original order.
 *   tts_render_fwd      per view: project and cull the survivors, build one
 *                       (tile id, mean vertex depth) key per overlapped tile,
 *                       sort the keys (Sec. 3.3: bucketed by tile, each tile's
 *                       list ordered by depth on chip), then per pixel blend the
 *                       tile's tets front to back with the Eq. 1 opacity of the
 *                       ray's chord through the tet and Eq. 2 compositing
 *                       (3DGS conventions), writing image, alpha and depth.
 *   tts_render_bwd      gradients of a scalar loss through the forward, given
 *                       dL/dimage, dL/dalpha, dL/ddepth: written to the vertex
 *                       positions, vertex SDF values and vertex colours.
 *   tts_render_fwd_ex / tts_render_bwd_ex
 *                       the same with the normal map of Eq. 2 as a fourth
 *                       channel (TTS_FLAG_NORMALS): N = sum_i T_i alpha_i n_i
 *                       with n_i the world-space unit gradient of tet i's
 *                       affine SDF (Sec. 3.2 "per-tetrahedron normal",
 *                       App. A.3), computed once per scene preparation.
 *
 * Everything runs on one CUDA device, asynchronously on the caller's stream.
 * No entry point allocates device memory: the caller provides one workspace
 * buffer sized by tts_workspace_size and keeps it (unchanged) from a forward
 * to the backward that follows it.
 *
 * Conventions
 *   camera     world->camera x_c = R v + t, R row-major, OpenCV axes (x right,
 *              y down, z forward); pixel (i, j) has its centre at
 *              (i + 0.5, j + 0.5) and sees the ray direction
 *              ((i + 0.5 - cx) / fx, (j + 0.5 - cy) / fy, 1).
 *   layouts    V: N x 3 fp32, T: K x 4 int32 (vertex indices), f: N fp32,
 *              rgb: N x 3 fp32, all contiguous.  Outputs are view-major and
 *              planar: view v occupies image[3 * P_v ...] as 3 planes of
 *              H_v x W_v, alpha[P_v ...] and depth[P_v ...] as H_v x W_v,
 *              where P_v = sum of H_u W_u over the views u < v.
 *   depth      Eq. 2 depth term: the blend of each tet's mean camera-space
 *              vertex depth z (not Euclidean distance).
 *   colour     each tet's colour is the mean of its four vertex colours.
 *   blending   alpha' = min(alpha, alpha_cap); fragments with alpha' <
 *              alpha_skip are skipped; a pixel stops before the fragment that
 *              would take its transmittance below t_eps; background is 0.
 *              With TTS_FLAG_PURE: no cap, no skip, no stop, no pre-filter.
 *
 * Errors: every call returns TTS_OK or a TTS_ERR_* code.  Argument errors are
 * found on the host before anything is enqueued.  Conditions found on the
 * device (an index outside [0, N), more keys than key_capacity, more
 * survivors than surv_capacity) set bits of a status word in the workspace;
 * tts_get_info reads it (and synchronises the stream).  When the status is not
 * zero the outputs of that forward/backward are undefined; enlarge the
 * capacities and call again.  Kernels never trap.
 */
#ifndef TETS_H_
#define TETS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tts_stream; /* a cudaStream_t (NULL: legacy default stream) */

enum {
  TTS_OK = 0,
  TTS_ERR_ARG = 1,        /* bad argument (host check) */
  TTS_ERR_WORKSPACE = 2,  /* workspace missing, misaligned or too small */
  TTS_ERR_OVERFLOW = 3,   /* status: key or survivor capacity exceeded */
  TTS_ERR_CUDA = 4,       /* a CUDA launch/runtime call failed */
  TTS_ERR_TIMEOUT = 5,    /* status: a bounded device wait gave up */
  TTS_ERR_BAD_INDEX = 6   /* status: a tet index outside [0, N) (tet dropped) */
};

/* status word bits (tts_info.status) */
enum {
  TTS_STATUS_BAD_INDEX = 1,
  TTS_STATUS_SURV_OVERFLOW = 2,
  TTS_STATUS_KEY_OVERFLOW = 4,
  TTS_STATUS_TIMEOUT = 8
};

enum {
  TTS_FLAG_PURE = 1,        /* no cap / skip / early stop / pre-filter */
  TTS_FLAG_ACCUM_GRAD = 2,  /* backward adds into dV/df/drgb instead of overwriting */
  TTS_FLAG_FORWARD_ONLY = 4, /* workspace without backward state; backward calls fail */
  TTS_FLAG_NORMALS = 8,      /* also render the normal map: use the _ex calls */
  TTS_FLAG_HULL = 16,        /* tile test against the projected tet (Sec. 3.3 culling): a tile
                                of a tet's bbox rect gets no key when, for some edge of the
                                convex hull of the four projected vertices, the corner pixel
                                centres of (tile x bbox) all lie strictly outside it (the exact
                                FP32 edge function fma(bu - au, pv - av, -((bv - av) * (pu - au)))
                                of hull edge (a, b) at corner p; rects of 2 to 2 x 2 tiles are
                                tested, others keep every tile) */
  TTS_FLAG_COUNT = 32        /* the blend kernels also count their walk (list groups scanned,
                                candidates staged, blocks walked): see
                                tts_debug_walk_counts; the result is unchanged */
};

#define TTS_MAX_SCENES 64
#define TTS_MAX_VIEWS 128

typedef struct {
  float R[9];     /* world -> camera rotation, row-major */
  float t[3];     /* world -> camera translation */
  float fx, fy, cx, cy;
  float znear;    /* a tet with any vertex at z < znear is culled */
  int32_t width, height;
} tts_camera;

typedef struct {
  float s;                /* Eq. 1 steepness */
  float prefilter_thresh; /* T_f, Sec. 3.2 (paper: 1/255) */
  float alpha_skip;       /* 1/255 */
  float alpha_cap;        /* 0.99 */
  float t_eps;            /* 1e-4 */
  int32_t tile;           /* tile edge in pixels: 8, 16 or 32 */
  int32_t flags;          /* TTS_FLAG_* */
  int32_t resort_window;  /* N_w of Sec. 3.3, 0..7: per pixel, fragments pass through a
                             window of N_w kept sorted by the depth of their chord's entry
                             point (ties: earlier first); the nearest leaves it when it holds
                             more than N_w, the rest at the end.  0: per-tile sort order. */
  int32_t blend_segment;  /* list entries per backward work unit: 0 (library default, 256)
                             or a multiple of 32 in 32..65536.  The forward walks each tile
                             list whole (a list longer than blend_segment as 4x2 blocks with
                             four lanes per pixel) and records its state every blend_segment
                             entries; the backward walks the segments of a longer list in
                             parallel from those states (equal to the unsplit walk up to
                             FP32 rounding).  Ignored with a resort window. */
  int32_t blend_warps;    /* warps per block of the persistent blend kernels: 0 (library
                             default, 4), 2, 4 or 8 (the resort-window kernels always use 4).
                             Changes the scheduling only, not the result. */
  int32_t frag_cap;       /* per-pixel fragment lists for the backward: 0 (library default,
                             128), 1..255, or -1 (none).  The forward records, per pixel, the
                             record slots of up to frag_cap blended fragments (4 bytes each:
                             frag_cap x 4 + 12 bytes of workspace per pixel) and a task list of
                             those pixels; the backward then takes each listed pixel with one
                             warp, one lane per fragment (transmittance and suffix by scans
                             over the lanes), and re-walks the tile lists only for tiles
                             holding a pixel with more blended fragments.  The same
                             arithmetic per fragment either way, up to rounding order.
                             Unused with a resort window, TTS_FLAG_FORWARD_ONLY or a batch of
                             2^32 pixels or more. */
} tts_params;

/* One scene: caller-owned device arrays (must outlive every call using them). */
typedef struct {
  const float* V;     /* N x 3 vertex positions */
  const int32_t* T;   /* K x 4 vertex indices */
  const float* f;     /* N vertex SDF values */
  const float* rgb;   /* N x 3 vertex colours */
  int64_t N, K;
  int64_t surv_capacity; /* record slots per view of this scene; 0 means K */
} tts_scene;

/* One view of one scene. */
typedef struct {
  tts_camera cam;
  int32_t scene;      /* index into the scene array */
  int32_t reserved;
} tts_view;

/* A batch: any number of scenes and views (up to the maxima above).  The
 * workspace layout is a pure function of (scenes' N, K, surv_capacity; views'
 * sizes and scenes; tile; flags; key_capacity). */
typedef struct {
  const tts_scene* scenes; /* host array */
  int32_t n_scenes;
  const tts_view* views;   /* host array */
  int32_t n_views;
  tts_params params;
  int64_t key_capacity;    /* (tile, tet) keys over all views */
  void* workspace;         /* device, 256-byte aligned */
  size_t workspace_bytes;
} tts_batch;

typedef struct {
  uint32_t status;          /* TTS_STATUS_* bits */
  int32_t n_scenes;
  int64_t n_keys;           /* keys produced by the last forward (needed capacity) */
  int64_t n_surv[TTS_MAX_SCENES]; /* survivors per scene of the last prepare */
  int32_t sort_bits;        /* bits of the (tile, depth) keys of the last forward */
  int32_t long_lists;       /* tiles of the last forward whose list exceeded the
                               on-chip sort of 4,096 keys (sorted by merging runs
                               in global memory) */
  int32_t blend_units;      /* blend work units (tile lists and list segments) */
  int32_t reserved;
} tts_info;

/* Bytes of workspace the batch needs (host only; nothing is enqueued). */
int tts_workspace_size(const tts_batch* b, size_t* bytes);

/* Clears the workspace's persistent state (status word, gradient
 * accumulators).  Call once after allocating or resizing the workspace. */
int tts_workspace_init(const tts_batch* b, tts_stream stream);

/* Pre-filter every scene of the batch (Sec. 3.2, view independent, hoisted
 * once per iteration as App. B.1 describes).  Writes the survivor lists into
 * the workspace. */
int tts_prepare_scene(const tts_batch* b, tts_stream stream);

/* Coarse-to-fine pre-filter (App. B.1), first round: the axis-aligned bounds
 * of the vertices of each scene's survivors of the last tts_prepare_scene.
 * aabb: device float[6 * n_scenes], (xmin, ymin, zmin, xmax, ymax, zmax) per
 * scene; a scene without survivors gets (+inf x3, -inf x3). */
int tts_survivor_bounds(const tts_batch* b, float* aabb, tts_stream stream);

/* Coarse-to-fine pre-filter, the resize between the rounds: maps the grid's
 * box [grid_lo, grid_hi] (host float[3] each) affinely, per axis, onto the
 * bounds aabb (device float[6], e.g. from tts_survivor_bounds) widened by
 * pad times its extent on each side: V_out = V_in * scale + offset
 * (N x 3, device; may alias V_in).  Empty bounds leave V_out = V_in.  The
 * caller then evaluates the SDF at the new vertices and prepares again. */
int tts_fit_grid(const float* V_in, int64_t N, const float grid_lo[3], const float grid_hi[3],
                 const float* aabb, float pad, float* V_out, tts_stream stream);

/* Forward for every view of the batch (needs tts_prepare_scene first).
 * image: 3 * sum(H W) floats, alpha and depth: sum(H W) floats (device). */
int tts_render_fwd(const tts_batch* b, float* image, float* alpha, float* depth,
                   tts_stream stream);

/* Outputs of a forward (device, layouts as above).  normal: 3 * sum(H W)
 * floats, planar like image; required with TTS_FLAG_NORMALS and NULL
 * without it (TTS_ERR_ARG otherwise). */
typedef struct {
  float* image;
  float* alpha;
  float* depth;
  float* normal;
} tts_outputs;

/* Upstream gradients of a backward (device, the layouts of tts_outputs).
 * dalpha, ddepth and dnormal may be NULL (zero); dnormal must be NULL
 * without TTS_FLAG_NORMALS. */
typedef struct {
  const float* dimage;
  const float* dalpha;
  const float* ddepth;
  const float* dnormal;
} tts_upstream;

/* tts_render_fwd with a tts_outputs (the only forward that can write the
 * normal map).  tts_render_fwd(b, i, a, d, s) equals this with normal NULL. */
int tts_render_fwd_ex(const tts_batch* b, const tts_outputs* out, tts_stream stream);

/* Backward of the last forward on this workspace.  dimage/dalpha/ddepth have
 * the layouts of the forward outputs; ddepth or dalpha may be NULL (zero).
 * dV, df, drgb: host arrays of n_scenes device pointers (N_s x 3, N_s,
 * N_s x 3 fp32), overwritten unless TTS_FLAG_ACCUM_GRAD. */
int tts_render_bwd(const tts_batch* b, const float* dimage, const float* dalpha,
                   const float* ddepth, float* const* dV, float* const* df,
                   float* const* drgb, tts_stream stream);

/* tts_render_bwd with a tts_upstream (adds dL/dnormal's contribution, which
 * reaches V and f through each tet's normal). */
int tts_render_bwd_ex(const tts_batch* b, const tts_upstream* up, float* const* dV,
                      float* const* df, float* const* drgb, tts_stream stream);

/* The forward and backward as their stages, for callers that interleave
 * their own work or time the stages: tts_render_fwd == tts_bin_views then
 * tts_blend_fwd; tts_render_bwd == tts_blend_bwd then tts_scatter_bwd (both
 * stages of a pair take the same batch).  tts_blend_bwd clears nothing:
 * tts_scatter_bwd overwrites (or, with TTS_FLAG_ACCUM_GRAD, adds into) the
 * vertex gradients. */
int tts_bin_views(const tts_batch* b, tts_stream stream);       /* cull, keys, sort, ranges */
int tts_blend_fwd(const tts_batch* b, float* image, float* alpha, float* depth,
                  tts_stream stream);                            /* per-tile blend */
int tts_blend_bwd(const tts_batch* b, const float* dimage, const float* dalpha,
                  const float* ddepth, tts_stream stream);       /* per-tile adjoint */
int tts_scatter_bwd(const tts_batch* b, float* const* dV, float* const* df,
                    float* const* drgb, tts_stream stream);      /* record -> vertex */
int tts_blend_fwd_ex(const tts_batch* b, const tts_outputs* out, tts_stream stream);
int tts_blend_bwd_ex(const tts_batch* b, const tts_upstream* up, tts_stream stream);

/* Number of kernels this library has launched in this process so far
 * (host-side counter, all threads). */
int64_t tts_launch_count(void);

/* Kernel-event hook, for timing the kernels of a call one by one: after
 * tts_debug_kernel_events(events, n) (events: n caller-created cudaEvent_t,
 * n <= 256), each kernel the library launches through its calls records the
 * next event on the call's stream right after the launch, until n have been
 * used.  tts_debug_kernel_events_used(names, max) returns how many were
 * recorded since the hook was set and fills names[i] (up to max) with the
 * name of the kernel the i-th event follows (strings owned by the CUDA
 * runtime).  n = 0 turns the hook off.  Process-wide, not thread safe,
 * returns TTS_ERR_ARG for n outside [0, 256] or missing events.  For
 * profiling: the events keep each kernel from overlapping the next. */
int tts_debug_kernel_events(void* const* events, int32_t n);
int32_t tts_debug_kernel_events_used(const char** names, int32_t max_names);

/* Test hook for the bounded waits of the binning's tile scan (a scan over
 * blocks of 2,048 tiles in which each block waits for the running sum of
 * the blocks before it).  spin_limit: polls of a predecessor's word before a
 * block gives up (0: the default, 2^22); unset_block: the index of a scan
 * block (in ticket order) whose wait polls a word that no block ever
 * publishes, so that it gives up after spin_limit polls (-1: none).  A wait
 * that gives up sets TTS_STATUS_TIMEOUT; that forward then uses no key (its
 * outputs are those of an empty scene) and the next forward clears the bit.
 * Process-wide, read when a call plans its launches; tts_debug_scan_wait(0,
 * -1) restores the defaults.  Returns TTS_ERR_ARG for spin_limit < 0 or
 * unset_block < -1.  Not for production use. */
int tts_debug_scan_wait(int64_t spin_limit, int32_t unset_block);

/* Device pointers to the per-pixel forward state (view-major, like alpha):
 * final transmittance (fp32), number of list entries walked up to the last
 * blended one (int32) and number of fragments met (int32: list entries whose
 * chord was non-empty, up to where the pixel stopped). */
int tts_debug_pixels(const tts_batch* b, const void** T_final, const void** last,
                     const void** n_frag, tts_stream stream);

/* Device pointers into the workspace to the per-pixel fragment lists of the
 * last forward (tts_params.frag_cap): *frag (uint32, frag_cap per pixel,
 * pixel-major: entry i of pixel p at p * frag_cap + i, the record slots of
 * the pixel's blended fragments in blend order), *n_blend (int32 per pixel:
 * its blended fragments, possibly more than the list holds) and *tile_over
 * (int32 per global tile: 1 when a pixel of the tile has more than frag_cap).
 * All three are null and *frag_cap is 0 when the batch keeps no lists.  Does
 * not launch or synchronise. */
int tts_debug_frag_lists(const tts_batch* b, const void** frag, const void** n_blend,
                         const void** tile_over, int32_t* frag_cap, tts_stream stream);

/* Walk statistics of the blend kernels since the last tts_workspace_init or
 * reset, accumulated by calls made with TTS_FLAG_COUNT (zero otherwise):
 * counts[0] the forward's list groups of 32 entries scanned, counts[1] list
 * entries it staged as candidates (their bbox meets a live pixel of the
 * warp's pixel block), counts[2] its pixel blocks walked; counts[3] and
 * counts[4] the groups and candidates of the list-walk backward (the
 * pixel-list backward's fragments are the blended counts of
 * tts_debug_frag_lists).  reset != 0 zeroes them after the copy.
 * Synchronises the stream. */
int tts_debug_walk_counts(const tts_batch* b, uint64_t counts[5], int32_t reset,
                          tts_stream stream);

/* Synchronises the stream and copies the status word and counters. */
int tts_get_info(const tts_batch* b, tts_info* info, tts_stream stream);

/* Device pointers into the workspace (for inspection and tests): the sorted
 * keys (uint64: (global tile << depth_bits) | (zbits - zmin_bits)), values
 * (uint32 record slot), per-tile ranges (int32 pairs [start, end) per global
 * tile), survivor list of scene 0.., and the key encoding (zmin_bits,
 * depth_bits).  A render keeps only the values and ranges: asking for keys
 * enqueues a kernel that rebuilds them into a scratch buffer of the workspace
 * from those and the slots' depth bits (valid until the next render).
 * Synchronises the stream. */
int tts_debug_lists(const tts_batch* b, const void** keys, const void** vals,
                    const void** ranges, const void** surv, uint32_t* zmin_bits,
                    int32_t* depth_bits, tts_stream stream);

/* Device pointer (*records) to the per-slot records of the last binning: 6
 * float4 per slot (pixel bbox with the front-face count in its signs, the
 * four face planes' P, A and B terms, the Eq. 1 field terms, mean depth and
 * colour); slot = the view's record base + survivor index.  A slot whose tet
 * is not visible in its view holds no defined record.  Does not launch or
 * synchronise; the pointer stays valid while the workspace does. */
int tts_debug_records(const tts_batch* b, const void** records, tts_stream stream);

/* Sorts n (key, value) pairs by the low key_bits bits of the key, stably
 * (bits above key_bits are carried along and take no part in the order): an
 * LSD radix sort with 8-bit digits (per pass: per-block digit counts, a scan
 * of the counts, a stable scatter), the device radix sort of Sec. 3.3's
 * (tile, depth) keys.  The binning of tts_bin_views does not call it: it
 * orders the same keys per tile on chip (a merge sort per tile list), with the
 * same result.  keys_in/vals_in (device, n each) are read only;
 * keys_out/vals_out receive the sorted pairs and must not alias the inputs.
 * scratch: device, 256-byte aligned, at least tts_sort_pairs_scratch_size(n)
 * bytes, owned by the caller, overwritten.  n <= 2^31 - 1.  Returns
 * TTS_ERR_ARG (bad n, key_bits outside [1, 64], aliasing) or
 * TTS_ERR_WORKSPACE (scratch missing, misaligned or too small) before
 * anything is enqueued, TTS_ERR_CUDA when one of its own kernel launches
 * failed (an error left pending by earlier unrelated CUDA calls is neither
 * reported nor cleared). */
int tts_sort_pairs_scratch_size(int64_t n, size_t* bytes);
int tts_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                   uint32_t* vals_out, int64_t n, int32_t key_bits, void* scratch,
                   size_t scratch_bytes, tts_stream stream);

/* The same sort without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory themselves (a custom allocator hook, which cannot
 * call back into cudaMalloc; plugin hosts that own every device allocation;
 * loops that cannot take cudaMalloc's implicit synchronisation).  keys_in/vals_in are
 * read only; keys_out/vals_out (device, n each) receive the sorted pairs and
 * must not alias the inputs.  Temporary storage is a fixed array of about
 * 12.3 MiB compiled into the library, present on every device that loads it
 * until the process exits, and shared by all calls: calls whose work overlaps
 * on the GPU race.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress); make it before any stream capture.  Returns
 * TTS_ERR_ARG for n > TTS_SORT_NOALLOC_MAX_KEYS, key_bits outside [1, 64] or
 * aliasing outputs, before anything is enqueued. */
#define TTS_SORT_NOALLOC_MAX_KEYS (1 << 20)
int tts_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                           uint32_t* vals_out, int64_t n, int32_t key_bits, tts_stream stream);

/* ------------------------------------------------------------------------
 * Geometry-stage terms (Sec. 4.2): the unique edges of a tet grid and the
 * eikonal and normal-consistency regularizers of its SDF.  Same conventions:
 * caller-owned device arrays and workspace (256-byte aligned), asynchronous
 * on the stream, argument errors found before anything is enqueued.  A tet or
 * edge with an index outside [0, N) is skipped and sets TTS_STATUS_BAD_INDEX
 * in the workspace's status word (tts_geometry_status).
 * ------------------------------------------------------------------------ */

/* Workspace bytes of tts_tet_edges for N vertices and K tets (6 K < 2^31). */
int tts_tet_edges_workspace_size(int64_t N, int64_t K, size_t* bytes);

/* The unique edges of the grid T (K x 4 int32, 16-byte aligned): the pairs
 * (lo, hi), lo < hi, of vertices that share a tet, sorted by (lo, hi).
 * edges: device int32 pairs (8-byte aligned), at most edge_capacity written
 * (6 K always suffices); *n_edges (device int64) receives the number of
 * edges, or -1 when an index was out of range. */
int tts_tet_edges(const int32_t* T, int64_t K, int64_t N, int32_t* edges, int64_t edge_capacity,
                  int64_t* n_edges, void* workspace, size_t workspace_bytes, tts_stream stream);

/* Workspace bytes of tts_regularizers for N vertices. */
int tts_regularizers_workspace_size(int64_t N, size_t* bytes);

/* Sec. 4.2 regularizers of the SDF f on the grid (V, T):
 *   L_eik = sum over tets k of (|g_k| - 1)^2, g_k the gradient of tet k's
 *           affine SDF (App. A.3);
 *   L_nc  = sum over the given edges (a, b) of 1 - cos(m_a, m_b), m_v the sum
 *           of the unit normals g_k / |g_k| of the tets containing v.
 * A flat tet (zero volume) contributes to neither; a tet with g = 0 adds 1 to
 * L_eik and nothing to m; an edge with m_a = 0 or m_b = 0 adds 1 to L_nc.
 * losses: device double[2] = (L_eik, L_nc), overwritten.  dV (N x 3), df (N):
 * device gradients of w_eik L_eik + w_nc L_nc, both NULL for losses only;
 * overwritten unless flags has TTS_FLAG_ACCUM_GRAD.  edges: E int32 pairs
 * (8-byte aligned), e.g. from tts_tet_edges. */
int tts_regularizers(const float* V, const int32_t* T, const float* f, int64_t N, int64_t K,
                     const int32_t* edges, int64_t E, float w_eik, float w_nc, double* losses,
                     float* dV, float* df, int32_t flags, void* workspace, size_t workspace_bytes,
                     tts_stream stream);

/* Workspace bytes of tts_marching_tets for K tets and E edges. */
int tts_marching_tets_workspace_size(int64_t K, int64_t E, size_t* bytes);

/* Marching Tetrahedra (Sec. 3.1, DMTet's extraction of the zero level set):
 * every edge of the sorted unique edge list (E pairs, e.g. from
 * tts_tet_edges) whose end points lie on different sides (positive: f > 0)
 * gets a vertex at the zero of the linear interpolation
 * (v_a f_b - v_b f_a) / (f_b - f_a); vertices are numbered in edge order.
 * Each tet with a 1-3 sign split gives one triangle (the cut edges of the odd
 * vertex o, in ascending order of the others' local index), each 2-2 tet two
 * (positive local vertices p < q, negative r < s: the quad pr, ps, qs, qr
 * split into (pr, ps, qs) and (pr, qs, qr)); triangles follow the tets in
 * order, wound so that their normal points towards increasing f (decided by
 * the sign of one FP32 vertex determinant per tet).
 * verts: device float (x, y, z) per vertex, vert_edge: its edge index
 * (nullable), at most vert_capacity written; tris: device int32 vertex index
 * triples, at most tri_capacity written.  counts: device int64[2] receives
 * (vertices, triangles) needed, so a call with zero capacities sizes the
 * outputs.  A tet edge missing from the list sets TTS_STATUS_BAD_INDEX. */
int tts_marching_tets(const float* V, const int32_t* T, const float* f, int64_t N, int64_t K,
                      const int32_t* edges, int64_t E, float* verts, int32_t* vert_edge,
                      int64_t vert_capacity, int32_t* tris, int64_t tri_capacity, int64_t* counts,
                      void* workspace, size_t workspace_bytes, tts_stream stream);

/* Synchronises the stream and reads the status word of a tts_tet_edges,
 * tts_regularizers or tts_marching_tets workspace. */
int tts_geometry_status(const void* workspace, uint32_t* status, tts_stream stream);

const char* tts_error_string(int code);

/* Library version and the GPU architecture it was built for. */
const char* tts_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TETS_H_ */
