// Geometry-stage terms of Sec. 4.2 on the GPU: the unique edges of a tet grid
// and the eikonal / normal-consistency regularizers of its SDF with their
// gradients.
//
// Edges: every tet emits its six (lo, hi) pairs into the bucket of lo
// (counting sort by lo), each bucket is sorted and deduplicated in place, and
// a scan of the per-vertex unique counts places the result, sorted by
// (lo, hi) whatever the order of the atomics.
//
// Regularizers (per call):
//   K_r1  per tet: g = h / det (App. A.3 through the cofactor columns),
//         (|g| - 1)^2 into L_eik (warp sums, one FP64 atomic per warp),
//         n = g / |g| added into the vertex sums m (FP32 atomics);
//   K_r2  per edge: 1 - cos(m_a, m_b) = |m_a/|m_a| - m_b/|m_b||^2 / 2 (no
//         cancellation near 1) into L_nc, and dL/dm at both ends;
//   K_r3  per tet: dL/dn = sum of dL/dm over its vertices, plus the eikonal
//         term, through g = h / det to dV and df (FP32 atomics).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "geo_common.cuh"

namespace tts {
namespace {

// ---------------------------------------------------------------------------
// edges
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RT) k_edge_count(const int4* __restrict__ T, long long K,
                                                   long long N, int* __restrict__ cnt,
                                                   GeoStatus* st) {
  bool bad = false;
  for (long long k = blockIdx.x * (long long)RT + threadIdx.x; k < K; k += (long long)gridDim.x * RT) {
    const int4 t = __ldg(T + k);
    if (!valid4(t, N)) { bad = true; continue; }
    const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int a = id[pair_a(e)], b = id[pair_b(e)];
      if (a != b) atomicAdd(cnt + min(a, b), 1);
    }
  }
  if (bad) atomicOr(&st->status, (unsigned)TTS_STATUS_BAD_INDEX);
}

__global__ void __launch_bounds__(RT) k_edge_fill(const int4* __restrict__ T, long long K,
                                                  long long N, const long long* __restrict__ off,
                                                  int* __restrict__ cur, int* __restrict__ bucket) {
  for (long long k = blockIdx.x * (long long)RT + threadIdx.x; k < K; k += (long long)gridDim.x * RT) {
    const int4 t = __ldg(T + k);
    if (!valid4(t, N)) continue;
    const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const int a = id[pair_a(e)], b = id[pair_b(e)];
      if (a == b) continue;
      const int lo = min(a, b);
      bucket[off[lo] + atomicAdd(cur + lo, 1)] = max(a, b);
    }
  }
}

// per vertex: insertion sort of its bucket, unique count
__global__ void __launch_bounds__(RT) k_edge_unique(long long N, const long long* __restrict__ off,
                                                    int* __restrict__ bucket,
                                                    int* __restrict__ ucnt) {
  for (long long v = blockIdx.x * (long long)RT + threadIdx.x; v < N; v += (long long)gridDim.x * RT) {
    const long long b0 = off[v], b1 = off[v + 1];
    for (long long i = b0 + 1; i < b1; ++i) {
      const int x = bucket[i];
      long long j = i - 1;
      while (j >= b0 && bucket[j] > x) {
        bucket[j + 1] = bucket[j];
        --j;
      }
      bucket[j + 1] = x;
    }
    int u = 0;
    for (long long i = b0; i < b1; ++i) u += (i == b0 || bucket[i] != bucket[i - 1]) ? 1 : 0;
    ucnt[v] = u;
  }
}

__global__ void __launch_bounds__(RT) k_edge_write(long long N, const long long* __restrict__ off,
                                                   const int* __restrict__ bucket,
                                                   const long long* __restrict__ uoff,
                                                   int2* __restrict__ edges, long long cap,
                                                   const GeoStatus* st, long long* n_edges) {
  for (long long v = blockIdx.x * (long long)RT + threadIdx.x; v < N; v += (long long)gridDim.x * RT) {
    long long o = uoff[v];
    const long long b0 = off[v], b1 = off[v + 1];
    for (long long i = b0; i < b1; ++i) {
      if (i == b0 || bucket[i] != bucket[i - 1]) {
        if (o < cap) edges[o] = make_int2((int)v, bucket[i]);
        ++o;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    *n_edges = (st->status & TTS_STATUS_BAD_INDEX) ? -1LL : st->total;
}

// ---------------------------------------------------------------------------
// regularizers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_vf(const float* __restrict__ V, const float* __restrict__ f,
                                        int4 t, float3 v[4], float fv[4]) {
  const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float* p = V + 3ll * id[j];
    v[j] = f3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
    fv[j] = __ldg(f + id[j]);
  }
}

__device__ __forceinline__ void warp_add_double(double x, double* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0 && x != 0.0) atomicAdd(dst, x);
}

__global__ void __launch_bounds__(RT) k_reg_tets(const float* __restrict__ V,
                                                 const int4* __restrict__ T,
                                                 const float* __restrict__ f, long long N,
                                                 long long K, float* __restrict__ m,
                                                 GeoStatus* st) {
  double le = 0.0;
  bool bad = false;
  const long long stride = (long long)gridDim.x * RT;
  const long long kend = (K + stride - 1) / stride * stride;   // whole warps reach the reduction
  for (long long k = blockIdx.x * (long long)RT + threadIdx.x; k < kend; k += stride) {
    if (k >= K) continue;
    const int4 t = __ldg(T + k);
    if (!valid4(t, N)) { bad = true; continue; }
    float3 v[4];
    float fv[4];
    load_vf(V, f, t, v, fv);
    TetGrad G;
    tet_grad(v, fv, G);
    if (G.det == 0.f) continue;                     // flat tet: no term
    const float gn = sqrtf(dot3(G.h, G.h)) / fabsf(G.det);
    le += (double)((gn - 1.f) * (gn - 1.f));
    float ih, sg;
    const float3 n = tet_unit_normal(G, &ih, &sg);
    if (ih == 0.f) continue;
    const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      atomicAdd(m + 3ll * id[j], n.x);
      atomicAdd(m + 3ll * id[j] + 1, n.y);
      atomicAdd(m + 3ll * id[j] + 2, n.z);
    }
  }
  warp_add_double(le, &st->acc[0]);
  if (bad) atomicOr(&st->status, (unsigned)TTS_STATUS_BAD_INDEX);
}

__global__ void __launch_bounds__(RT) k_reg_edges(const int2* __restrict__ edges, long long E,
                                                  long long N, const float* __restrict__ m,
                                                  float w_nc, float* __restrict__ dm,
                                                  GeoStatus* st) {
  double ln = 0.0;
  bool bad = false;
  const long long stride = (long long)gridDim.x * RT;
  const long long eend = (E + stride - 1) / stride * stride;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < eend; e += stride) {
    if (e >= E) continue;
    const int2 ab = __ldg(edges + e);
    if ((unsigned long long)ab.x >= (unsigned long long)N ||
        (unsigned long long)ab.y >= (unsigned long long)N) { bad = true; continue; }
    const float3 ma = f3(m[3ll * ab.x], m[3ll * ab.x + 1], m[3ll * ab.x + 2]);
    const float3 mb = f3(m[3ll * ab.y], m[3ll * ab.y + 1], m[3ll * ab.y + 2]);
    const float na = sqrtf(dot3(ma, ma)), nb = sqrtf(dot3(mb, mb));
    if (!(na > 0.f && nb > 0.f)) {
      ln += 1.0;
      continue;
    }
    const float3 ua = (1.f / na) * ma, ub = (1.f / nb) * mb;
    const float3 d = ua - ub;
    ln += 0.5 * (double)dot3(d, d);
    if (dm) {
      const float cs = dot3(ua, ub);
      // d(1 - cos)/d m_a = -(u_b - cos u_a) / |m_a|
      const float3 ga = (-w_nc / na) * (ub - cs * ua);
      const float3 gb = (-w_nc / nb) * (ua - cs * ub);
      atomicAdd(dm + 3ll * ab.x, ga.x);
      atomicAdd(dm + 3ll * ab.x + 1, ga.y);
      atomicAdd(dm + 3ll * ab.x + 2, ga.z);
      atomicAdd(dm + 3ll * ab.y, gb.x);
      atomicAdd(dm + 3ll * ab.y + 1, gb.y);
      atomicAdd(dm + 3ll * ab.y + 2, gb.z);
    }
  }
  warp_add_double(ln, &st->acc[1]);
  if (bad) atomicOr(&st->status, (unsigned)TTS_STATUS_BAD_INDEX);
}

__global__ void __launch_bounds__(RT) k_reg_tets_bwd(const float* __restrict__ V,
                                                     const int4* __restrict__ T,
                                                     const float* __restrict__ f, long long N,
                                                     long long K, const float* __restrict__ dm,
                                                     float w_eik, float* __restrict__ dV,
                                                     float* __restrict__ df) {
  for (long long k = blockIdx.x * (long long)RT + threadIdx.x; k < K; k += (long long)gridDim.x * RT) {
    const int4 t = __ldg(T + k);
    if (!valid4(t, N)) continue;
    float3 v[4];
    float fv[4];
    load_vf(V, f, t, v, fv);
    TetGrad G;
    tet_grad(v, fv, G);
    if (G.det == 0.f) continue;
    float ih, sg;
    const float3 n = tet_unit_normal(G, &ih, &sg);
    if (ih == 0.f) continue;                        // g = 0: no gradient
    const int id[4] = {t.x, t.y, t.z, t.w};
    float3 dn = f3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      dn = dn + f3(dm[3ll * id[j]], dm[3ll * id[j] + 1], dm[3ll * id[j] + 2]);
    const float idet = 1.f / G.det;
    const float gn = sqrtf(dot3(G.h, G.h)) * fabsf(idet);
    // dL/dg: eikonal 2 (|g| - 1) n, normal consistency (I - n n^T) dn / |g|
    const float3 dg = (2.f * w_eik * (gn - 1.f)) * n + (1.f / gn) * (dn - dot3(n, dn) * n);
    // g = h / det
    const float3 g = idet * G.h;
    float3 dv[4] = {f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0)};
    float dfv[4] = {0.f, 0.f, 0.f, 0.f};
    tet_grad_adjoint(G, idet * dg, -dot3(dg, g) * idet, dv, dfv);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      atomicAdd(dV + 3ll * id[j], dv[j].x);
      atomicAdd(dV + 3ll * id[j] + 1, dv[j].y);
      atomicAdd(dV + 3ll * id[j] + 2, dv[j].z);
      atomicAdd(df + id[j], dfv[j]);
    }
  }
}

__global__ void k_reg_finish(const GeoStatus* st, double* losses) {
  losses[0] = st->acc[0];
  losses[1] = st->acc[1];
}

struct EdgeWs {
  size_t bytes;
  size_t o_st, o_cnt, o_off, o_sums, o_bucket, o_ucnt, o_uoff, o_usums;
};

EdgeWs edge_layout(long long N, long long K) {
  EdgeWs w;
  size_t off = 0;
  auto take = [&](size_t b) { off = align256(off); const size_t r = off; off += b; return r; };
  const long long nb = (N + SCAN_CHUNK - 1) / SCAN_CHUNK;
  w.o_st = take(sizeof(GeoStatus));
  w.o_cnt = take(sizeof(int) * N);
  w.o_off = take(sizeof(long long) * (N + 1));
  w.o_sums = take(sizeof(long long) * nb);
  w.o_bucket = take(sizeof(int) * 6 * K);
  w.o_ucnt = take(sizeof(int) * N);
  w.o_uoff = take(sizeof(long long) * (N + 1));
  w.o_usums = take(sizeof(long long) * nb);
  w.bytes = align256(off);
  return w;
}

struct RegWs {
  size_t bytes;
  size_t o_st, o_m, o_dm;
};

RegWs reg_layout(long long N) {
  RegWs w;
  size_t off = 0;
  auto take = [&](size_t b) { off = align256(off); const size_t r = off; off += b; return r; };
  w.o_st = take(sizeof(GeoStatus));
  w.o_m = take(sizeof(float) * 3 * N);
  w.o_dm = take(sizeof(float) * 3 * N);
  w.bytes = align256(off);
  return w;
}

}  // namespace

}  // namespace tts

using namespace tts;

extern "C" {

int tts_tet_edges_workspace_size(int64_t N, int64_t K, size_t* bytes) {
  if (!bytes || !sizes_ok(N, K)) return TTS_ERR_ARG;
  *bytes = edge_layout(N, K).bytes;
  return TTS_OK;
}

int tts_tet_edges(const int32_t* T, int64_t K, int64_t N, int32_t* edges, int64_t edge_capacity,
                  int64_t* n_edges, void* workspace, size_t workspace_bytes, tts_stream stream) {
  if (!T || !edges || !n_edges || !sizes_ok(N, K) || edge_capacity < 0) return TTS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(T) % 16 != 0 || reinterpret_cast<uintptr_t>(edges) % 8 != 0)
    return TTS_ERR_ARG;
  const EdgeWs w = edge_layout(N, K);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 != 0 || workspace_bytes < w.bytes)
    return TTS_ERR_WORKSPACE;
  char* base = static_cast<char*>(workspace);
  GeoStatus* st = reinterpret_cast<GeoStatus*>(base + w.o_st);
  int* cnt = reinterpret_cast<int*>(base + w.o_cnt);
  long long* off = reinterpret_cast<long long*>(base + w.o_off);
  long long* sums = reinterpret_cast<long long*>(base + w.o_sums);
  int* bucket = reinterpret_cast<int*>(base + w.o_bucket);
  int* ucnt = reinterpret_cast<int*>(base + w.o_ucnt);
  long long* uoff = reinterpret_cast<long long*>(base + w.o_uoff);
  long long* usums = reinterpret_cast<long long*>(base + w.o_usums);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int4* T4 = reinterpret_cast<const int4*>(T);
  if (cudaMemsetAsync(st, 0, sizeof(GeoStatus), s) != cudaSuccess ||
      cudaMemsetAsync(cnt, 0, sizeof(int) * N, s) != cudaSuccess)
    return TTS_ERR_CUDA;
  long long n = 0;
  k_edge_count<<<grid_for(K), RT, 0, s>>>(T4, K, N, cnt, st);
  n += 1 + scan_counts(cnt, N, sums, off, &st->total, s);
  if (cudaMemsetAsync(cnt, 0, sizeof(int) * N, s) != cudaSuccess) return TTS_ERR_CUDA;
  k_edge_fill<<<grid_for(K), RT, 0, s>>>(T4, K, N, off, cnt, bucket);
  k_edge_unique<<<grid_for(N), RT, 0, s>>>(N, off, bucket, ucnt);
  n += 2 + scan_counts(ucnt, N, usums, uoff, &st->total, s);
  k_edge_write<<<grid_for(N), RT, 0, s>>>(N, off, bucket, uoff, reinterpret_cast<int2*>(edges),
                                          edge_capacity, st, reinterpret_cast<long long*>(n_edges));
  count_launches(n + 1);
  return (cudaPeekAtLastError() == cudaSuccess) ? TTS_OK : TTS_ERR_CUDA;
}

int tts_regularizers_workspace_size(int64_t N, size_t* bytes) {
  if (!bytes || N < 1 || N > 0x7fffffffLL) return TTS_ERR_ARG;
  *bytes = reg_layout(N).bytes;
  return TTS_OK;
}

int tts_regularizers(const float* V, const int32_t* T, const float* f, int64_t N, int64_t K,
                     const int32_t* edges, int64_t E, float w_eik, float w_nc, double* losses,
                     float* dV, float* df, int32_t flags, void* workspace, size_t workspace_bytes,
                     tts_stream stream) {
  if (!V || !T || !f || !losses || !sizes_ok(N, K) || E < 0 || (E > 0 && !edges)) return TTS_ERR_ARG;
  if ((dV == nullptr) != (df == nullptr)) return TTS_ERR_ARG;
  if (!(std::isfinite(w_eik) && std::isfinite(w_nc))) return TTS_ERR_ARG;
  if (flags & ~TTS_FLAG_ACCUM_GRAD) return TTS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(T) % 16 != 0 || (E > 0 && reinterpret_cast<uintptr_t>(edges) % 8 != 0))
    return TTS_ERR_ARG;
  const RegWs w = reg_layout(N);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 != 0 || workspace_bytes < w.bytes)
    return TTS_ERR_WORKSPACE;
  char* base = static_cast<char*>(workspace);
  GeoStatus* st = reinterpret_cast<GeoStatus*>(base + w.o_st);
  float* m = reinterpret_cast<float*>(base + w.o_m);
  float* dm = reinterpret_cast<float*>(base + w.o_dm);
  const bool grad = dV != nullptr;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int4* T4 = reinterpret_cast<const int4*>(T);
  const int2* E2 = reinterpret_cast<const int2*>(edges);
  if (cudaMemsetAsync(st, 0, sizeof(GeoStatus), s) != cudaSuccess ||
      cudaMemsetAsync(m, 0, sizeof(float) * 3 * N, s) != cudaSuccess)
    return TTS_ERR_CUDA;
  if (grad) {
    if (cudaMemsetAsync(dm, 0, sizeof(float) * 3 * N, s) != cudaSuccess) return TTS_ERR_CUDA;
    if (!(flags & TTS_FLAG_ACCUM_GRAD) &&
        (cudaMemsetAsync(dV, 0, sizeof(float) * 3 * N, s) != cudaSuccess ||
         cudaMemsetAsync(df, 0, sizeof(float) * N, s) != cudaSuccess))
      return TTS_ERR_CUDA;
  }
  long long n = 0;
  k_reg_tets<<<grid_for(K), RT, 0, s>>>(V, T4, f, N, K, m, st);
  ++n;
  if (E > 0) {
    k_reg_edges<<<grid_for(E), RT, 0, s>>>(E2, E, N, m, w_nc, grad ? dm : nullptr, st);
    ++n;
  }
  if (grad) {
    k_reg_tets_bwd<<<grid_for(K), RT, 0, s>>>(V, T4, f, N, K, dm, w_eik, dV, df);
    ++n;
  }
  k_reg_finish<<<1, 1, 0, s>>>(st, losses);
  count_launches(n + 1);
  return (cudaPeekAtLastError() == cudaSuccess) ? TTS_OK : TTS_ERR_CUDA;
}

int tts_geometry_status(const void* workspace, uint32_t* status, tts_stream stream) {
  if (!workspace || !status || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return TTS_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GeoStatus h;
  if (cudaMemcpyAsync(&h, workspace, sizeof(GeoStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TTS_ERR_CUDA;
  *status = h.status;
  return TTS_OK;
}

}  // extern "C"
