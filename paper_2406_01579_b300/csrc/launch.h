// Host-side launch plan shared by the kernel translation units and the API.
#pragma once

#include <cuda_runtime.h>

#include "tets_internal.cuh"

namespace tts {

struct HostPlan {
  int n_scenes, n_views;
  int max_pf_chunks, max_pp_chunks, max_pre_chunks;
  int tsort_blocks;         // persistent grid of the depth sort
  int wl_blocks;
  int total_tiles;
  int tile;
  int window;
  bool normals;
  bool hull;                // tile test against the projected tet (TTS_FLAG_HULL)
  int normal_blocks;
  int tet_bwd_blocks;
  int blend_fwd_blocks, blend_bwd_blocks;
  int blend_warps;          // warps per block of the main blend kernels (2, 4 or 8)
  int frag_cap;             // per-pixel fragment list capacity (0: no lists)
  bool count;               // TTS_FLAG_COUNT: the counting instantiation of the forward
  unsigned* px_clear;       // device address of Counters::px_n and ::ovf_any (cleared per forward)
  int px_blocks;            // grid of the pixel-list backward (grid stride over the listed pixels)
  long long total_pixels;
};

struct GradOut {
  float* dV[TTS_MAX_SCENES];
  float* df[TTS_MAX_SCENES];
  float* drgb[TTS_MAX_SCENES];
};

// Launch with programmatic stream serialization (see pdl_wait): the kernel's
// blocks may be scheduled while the previous kernel in the stream finishes.
// A launch error is kept for check_launch.  With the kernel-event hook on
// (tts_debug_kernel_events), an event is recorded after the launch.
void note_launch_error(cudaError_t e);
void note_kernel_launched(const void* kernel, cudaStream_t st);
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e != cudaSuccess) note_launch_error(e);
  note_kernel_launched(reinterpret_cast<const void*>(kernel), st);
}

// Each launcher returns the number of kernels it launched.
int launch_prefilter(const HostPlan& P, const Batch* dB, cudaStream_t st);
int launch_binning(const HostPlan& P, const Batch* dB, cudaStream_t st);
int launch_debug_keys(const HostPlan& P, const Batch* dB, cudaStream_t st);
int launch_bounds(const HostPlan& P, const Batch* dB, float* aabb, cudaStream_t st);
int launch_fit_grid(const float* V_in, long long N, const float lo[3], const float hi[3],
                    const float* aabb, float pad, float* V_out, cudaStream_t st);
int launch_blend_fwd(const HostPlan& P, const Batch* dB, float* image, float* alpha, float* depth,
                     float* normal, cudaStream_t st);
int px_grid(int tile, bool normals, int sms);
int launch_blend_bwd(const HostPlan& P, const Batch* dB, const float* dimage, const float* dalpha,
                     const float* ddepth, const float* dnormal, const GradOut* zero,
                     cudaStream_t st);
int launch_tet_bwd(const HostPlan& P, const Batch* dB, const GradOut& go, cudaStream_t st);
int launch_zero_grads(const HostPlan& P, const Batch* dB, const GradOut& go, cudaStream_t st);
int launch_upload(const Batch& hb, Batch* dB, cudaStream_t st);
// persistent grid sizes of the blend kernels for a tile size (occupancy based)
void blend_grid(int tile, bool normals, int window, int warps, int sms, int* fwd_blocks,
                int* bwd_blocks);

}  // namespace tts
