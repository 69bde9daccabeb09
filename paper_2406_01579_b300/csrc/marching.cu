// Marching Tetrahedra on the GPU (Sec. 3.1: the representation keeps DMTet's
// mesh extraction).  Given the grid's sorted unique edges:
//   K_m1  per edge: does it cross the zero level set (positive: f > 0)?
//   scan  crossing flags -> vertex index per crossing edge (edge order)
//   K_m2  per crossing edge: the zero of the linear interpolation
//   K_m3  per tet: 0, 1 (1-3 sign split) or 2 (2-2 split) triangles
//   scan  triangle counts -> triangle offset per tet (tet order)
//   K_m4  per cut tet: its crossing edges' vertex indices by binary search in
//         the edge list, triangles wound so that the normal points towards
//         increasing f (the sign of one vertex determinant decides).
// Output order is fixed by the two scans, independent of scheduling.
#include <cmath>

#include "geo_common.cuh"

namespace tts {
namespace {

__global__ void __launch_bounds__(RT) k_mt_edge_flag(const int2* __restrict__ edges, long long E,
                                                     long long N, const float* __restrict__ f,
                                                     int* __restrict__ flag, GeoStatus* st) {
  bool bad = false;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < E; e += (long long)gridDim.x * RT) {
    const int2 ab = __ldg(edges + e);
    int c = 0;
    if ((unsigned long long)ab.x < (unsigned long long)N &&
        (unsigned long long)ab.y < (unsigned long long)N)
      c = ((__ldg(f + ab.x) > 0.f) != (__ldg(f + ab.y) > 0.f)) ? 1 : 0;
    else
      bad = true;
    flag[e] = c;
  }
  if (bad) atomicOr(&st->status, (unsigned)TTS_STATUS_BAD_INDEX);
}

__global__ void __launch_bounds__(RT) k_mt_verts(const float* __restrict__ V,
                                                 const float* __restrict__ f,
                                                 const int2* __restrict__ edges, long long E,
                                                 const int* __restrict__ flag,
                                                 const long long* __restrict__ voff,
                                                 float* __restrict__ verts,
                                                 int* __restrict__ vert_edge, long long vcap) {
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < E; e += (long long)gridDim.x * RT) {
    if (!flag[e]) continue;
    const long long o = voff[e];
    if (o >= vcap) continue;
    const int2 ab = __ldg(edges + e);
    const float fa = __ldg(f + ab.x), fb = __ldg(f + ab.y);
    const float den = fb - fa;     // |fa| + |fb| > 0: the signs differ
#pragma unroll
    for (int r = 0; r < 3; ++r)
      verts[3 * o + r] = (__ldg(V + 3ll * ab.x + r) * fb - __ldg(V + 3ll * ab.y + r) * fa) / den;
    if (vert_edge) vert_edge[o] = (int)e;
  }
}

__device__ __forceinline__ int tet_case(const float fv[4], int* np) {
  int m = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) m |= (fv[i] > 0.f) ? (1 << i) : 0;
  *np = __popc(m);
  return m;
}

__global__ void __launch_bounds__(RT) k_mt_tet_count(const int4* __restrict__ T, long long K,
                                                     long long N, const float* __restrict__ f,
                                                     int* __restrict__ cnt, GeoStatus* st) {
  bool bad = false;
  for (long long k = blockIdx.x * (long long)RT + threadIdx.x; k < K; k += (long long)gridDim.x * RT) {
    const int4 t = __ldg(T + k);
    int c = 0;
    if (valid4(t, N)) {
      const float fv[4] = {__ldg(f + t.x), __ldg(f + t.y), __ldg(f + t.z), __ldg(f + t.w)};
      int np;
      tet_case(fv, &np);
      c = (np == 1 || np == 3) ? 1 : (np == 2 ? 2 : 0);
    } else {
      bad = true;
    }
    cnt[k] = c;
  }
  if (bad) atomicOr(&st->status, (unsigned)TTS_STATUS_BAD_INDEX);
}

// index of the edge (min(x,y), max(x,y)) in the sorted list, or -1
__device__ __forceinline__ long long find_edge(const int2* __restrict__ edges, long long E, int x,
                                               int y) {
  const unsigned long long key = ((unsigned long long)(unsigned)min(x, y) << 32) | (unsigned)max(x, y);
  long long lo = 0, hi = E;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    const int2 m = __ldg(edges + mid);
    const unsigned long long mk = ((unsigned long long)(unsigned)m.x << 32) | (unsigned)m.y;
    if (mk < key) lo = mid + 1; else hi = mid;
  }
  if (lo < E) {
    const int2 m = __ldg(edges + lo);
    if (m.x == min(x, y) && m.y == max(x, y)) return lo;
  }
  return -1;
}

__device__ __forceinline__ float det3(float3 o, float3 a, float3 b, float3 c) {
  return dot3(a - o, cross3(b - o, c - o));
}

__global__ void __launch_bounds__(RT) k_mt_tris(const float* __restrict__ V,
                                                const int4* __restrict__ T, long long K,
                                                const float* __restrict__ f,
                                                const int2* __restrict__ edges, long long E,
                                                const long long* __restrict__ voff,
                                                const int* __restrict__ cnt,
                                                const long long* __restrict__ toff,
                                                int* __restrict__ tris, long long tcap,
                                                GeoStatus* st) {
  bool missing = false;
  for (long long k = blockIdx.x * (long long)RT + threadIdx.x; k < K; k += (long long)gridDim.x * RT) {
    if (cnt[k] == 0) continue;
    const int4 t = __ldg(T + k);
    const int id[4] = {t.x, t.y, t.z, t.w};
    float fv[4];
    float3 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      fv[i] = __ldg(f + id[i]);
      p[i] = f3(__ldg(V + 3ll * id[i]), __ldg(V + 3ll * id[i] + 1), __ldg(V + 3ll * id[i] + 2));
    }
    int np;
    const int m = tet_case(fv, &np);
    const long long o = toff[k];
    // local vertex order: the odd / positive ones first, each group ascending
    int a[4], na = 0, nb = 0, b[4];
    const bool odd_pos = (np == 1) || (np == 2);   // group A = positive for 1 and 2, negative for 3
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool pos = (m >> i) & 1;
      if (pos == odd_pos) a[na++] = i; else b[nb++] = i;
    }
    auto vid = [&](int i, int j) -> long long {
      const long long e = find_edge(edges, E, id[i], id[j]);
      if (e < 0) { missing = true; return 0; }
      return voff[e];
    };
    if (np == 1 || np == 3) {
      const int ov = a[0];
      const long long x = vid(ov, b[0]), y = vid(ov, b[1]), z = vid(ov, b[2]);
      const float D = det3(p[ov], p[b[0]], p[b[1]], p[b[2]]);
      const bool flip = (np == 1) ? (D > 0.f) : (D < 0.f);
      if (o < tcap) {
        tris[3 * o] = (int)x;
        tris[3 * o + 1] = (int)(flip ? z : y);
        tris[3 * o + 2] = (int)(flip ? y : z);
      }
    } else {
      const int pp = a[0], q = a[1], r = b[0], s = b[1];
      const long long pr = vid(pp, r), ps = vid(pp, s), qs = vid(q, s), qr = vid(q, r);
      const float D = det3(p[pp], p[q], p[r], p[s]);
      const bool flip = D > 0.f;
      if (o < tcap) {
        tris[3 * o] = (int)pr;
        tris[3 * o + 1] = (int)(flip ? qs : ps);
        tris[3 * o + 2] = (int)(flip ? ps : qs);
      }
      if (o + 1 < tcap) {
        tris[3 * o + 3] = (int)pr;
        tris[3 * o + 4] = (int)(flip ? qr : qs);
        tris[3 * o + 5] = (int)(flip ? qs : qr);
      }
    }
  }
  if (missing) atomicOr(&st->status, (unsigned)TTS_STATUS_BAD_INDEX);
}

__global__ void k_mt_finish(const GeoStatus* st, long long* counts) {
  counts[0] = st->counts[0];
  counts[1] = st->counts[1];
}

struct MtWs {
  size_t bytes;
  size_t o_st, o_eflag, o_voff, o_esums, o_tcnt, o_toff, o_tsums;
};

MtWs mt_layout(long long K, long long E) {
  MtWs w;
  size_t off = 0;
  auto take = [&](size_t b) { off = align256(off); const size_t r = off; off += b; return r; };
  const long long nbe = (E + SCAN_CHUNK - 1) / SCAN_CHUNK, nbk = (K + SCAN_CHUNK - 1) / SCAN_CHUNK;
  w.o_st = take(sizeof(GeoStatus));
  w.o_eflag = take(sizeof(int) * E);
  w.o_voff = take(sizeof(long long) * (E + 1));
  w.o_esums = take(sizeof(long long) * std::max(1LL, nbe));
  w.o_tcnt = take(sizeof(int) * K);
  w.o_toff = take(sizeof(long long) * (K + 1));
  w.o_tsums = take(sizeof(long long) * nbk);
  w.bytes = align256(off);
  return w;
}

}  // namespace
}  // namespace tts

using namespace tts;

extern "C" {

int tts_marching_tets_workspace_size(int64_t K, int64_t E, size_t* bytes) {
  if (!bytes || K < 1 || E < 1 || 6 * K > 0x7fffffffLL || E > 6 * K) return TTS_ERR_ARG;
  *bytes = mt_layout(K, E).bytes;
  return TTS_OK;
}

int tts_marching_tets(const float* V, const int32_t* T, const float* f, int64_t N, int64_t K,
                      const int32_t* edges, int64_t E, float* verts, int32_t* vert_edge,
                      int64_t vert_capacity, int32_t* tris, int64_t tri_capacity, int64_t* counts,
                      void* workspace, size_t workspace_bytes, tts_stream stream) {
  if (!V || !T || !f || !edges || !verts || !tris || !counts || !sizes_ok(N, K)) return TTS_ERR_ARG;
  if (E < 1 || E > 6 * K || vert_capacity < 0 || tri_capacity < 0) return TTS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(T) % 16 != 0 || reinterpret_cast<uintptr_t>(edges) % 8 != 0)
    return TTS_ERR_ARG;
  const MtWs w = mt_layout(K, E);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 != 0 || workspace_bytes < w.bytes)
    return TTS_ERR_WORKSPACE;
  char* base = static_cast<char*>(workspace);
  GeoStatus* st = reinterpret_cast<GeoStatus*>(base + w.o_st);
  int* eflag = reinterpret_cast<int*>(base + w.o_eflag);
  long long* voff = reinterpret_cast<long long*>(base + w.o_voff);
  long long* esums = reinterpret_cast<long long*>(base + w.o_esums);
  int* tcnt = reinterpret_cast<int*>(base + w.o_tcnt);
  long long* toff = reinterpret_cast<long long*>(base + w.o_toff);
  long long* tsums = reinterpret_cast<long long*>(base + w.o_tsums);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int4* T4 = reinterpret_cast<const int4*>(T);
  const int2* E2 = reinterpret_cast<const int2*>(edges);
  if (cudaMemsetAsync(st, 0, sizeof(GeoStatus), s) != cudaSuccess) return TTS_ERR_CUDA;
  long long n = 0;
  k_mt_edge_flag<<<grid_for(E), RT, 0, s>>>(E2, E, N, f, eflag, st);
  n += 1 + scan_counts(eflag, E, esums, voff, &st->counts[0], s);
  k_mt_verts<<<grid_for(E), RT, 0, s>>>(V, f, E2, E, eflag, voff, verts, vert_edge, vert_capacity);
  k_mt_tet_count<<<grid_for(K), RT, 0, s>>>(T4, K, N, f, tcnt, st);
  n += 2 + scan_counts(tcnt, K, tsums, toff, &st->counts[1], s);
  k_mt_tris<<<grid_for(K), RT, 0, s>>>(V, T4, K, f, E2, E, voff, tcnt, toff, tris, tri_capacity, st);
  k_mt_finish<<<1, 1, 0, s>>>(st, reinterpret_cast<long long*>(counts));
  count_launches(n + 2);
  return (cudaPeekAtLastError() == cudaSuccess) ? TTS_OK : TTS_ERR_CUDA;
}

}  // extern "C"
