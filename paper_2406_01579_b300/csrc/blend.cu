// Per-tile blending (Eq. 1 opacity of each pixel's chord, Eq. 2 compositing
// with the 3DGS conventions), its backward, and the record -> vertex adjoint.
#include "geometry.cuh"
#include "launch.h"

namespace tts {

constexpr int BLEND_BATCH = 256;   // records staged in shared memory per round

__device__ __forceinline__ int find_view(const Batch* __restrict__ B, int gt) {
  int lo = 0, hi = B->n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B->vw[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Pixel of this thread inside the tile: warps cover 8x4 pixel blocks.
template <int TILE>
struct PixelMap {
  int px, py;
  float wx0, wx1, wy0, wy1;  // warp's pixel-centre rectangle
  __device__ __forceinline__ PixelMap(int txi, int tyi) {
    constexpr int WX = TILE / 8;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wx = wid % WX, wy = wid / WX;
    const int bx = txi * TILE + wx * 8, by = tyi * TILE + wy * 4;
    px = bx + (lane & 7);
    py = by + (lane >> 3);
    wx0 = (float)bx + 0.5f;
    wx1 = wx0 + 7.f;
    wy0 = (float)by + 0.5f;
    wy1 = wy0 + 3.f;
  }
  __device__ __forceinline__ bool warp_misses(const float4& q0) const {
    return (fabsf(q0.x) > wx1) | (q0.z < wx0) | (fabsf(q0.y) > wy1) | (q0.w < wy0);
  }
};

// ---------------------------------------------------------------------------
// K6: forward blend.  One CTA per (view, tile), one thread per pixel.
// ---------------------------------------------------------------------------
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_blend_fwd(const Batch* __restrict__ B,
                                                           float* __restrict__ image,
                                                           float* __restrict__ alpha,
                                                           float* __restrict__ depth) {
  constexpr int NT = TILE * TILE;
  __shared__ float4 sm[REC_Q][BLEND_BATCH];
  const int gt = blockIdx.x;
  const ViewD& vw = B->vw[find_view(B, gt)];
  const int lt = gt - vw.tile_base;
  const int tyi = lt / vw.tiles_x, txi = lt - tyi * vw.tiles_x;
  const PixelMap<TILE> pm(txi, tyi);
  const bool inimg = (pm.px < vw.W) & (pm.py < vw.H);
  const float fpx = (float)pm.px + 0.5f, fpy = (float)pm.py + 0.5f;
  const Counters* c = B->ctr;
  const int2 rg = B->ranges[gt];
  const unsigned* __restrict__ vals = B->vals[c->n_passes & 1];
  const float4* __restrict__ rec = B->rec;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap, skip = B->alpha_skip, eps = B->t_eps;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  int last = 0, nfrag = 0;
  bool done = !inimg;
  for (int base = rg.x; base < rg.y; base += BLEND_BATCH) {
    if (__syncthreads_count(!done) == 0) break;
    const int n = min(BLEND_BATCH, rg.y - base);
    for (int i = threadIdx.x; i < n; i += NT) {
      const float4* r = rec + (size_t)vals[base + i] * REC_Q;
#pragma unroll
      for (int q = 0; q < REC_Q; ++q) sm[q][i] = __ldg(r + q);
    }
    __syncthreads();
    if (!done) {
      for (int j = 0; j < n; ++j) {
        const float4 q0 = sm[0][j];
        if (pm.warp_misses(q0)) continue;
        const Chord ch = chord_eval(q0, sm[1][j], sm[2][j], sm[3][j], fpx, fpy);
        if (!ch.hit) continue;
        ++nfrag;
        const Opacity o = opacity_eval(sm[4][j], ch);
        float a = o.alpha;
        if (!pure) {
          a = fminf(a, cap);
          if (a < skip) continue;
        } else if (!(a > 0.f)) {
          continue;
        }
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
        if (!pure && Tn < eps) { done = true; break; }
        const float4 q5 = sm[5][j];
        const float wgt = __fmul_rn(T, a);
        C0 = __fmaf_rn(wgt, q5.y, C0);
        C1 = __fmaf_rn(wgt, q5.z, C1);
        C2 = __fmaf_rn(wgt, q5.w, C2);
        D = __fmaf_rn(wgt, q5.x, D);
        T = Tn;
        last = base + j - rg.x + 1;
      }
    }
  }
  if (inimg) {
    const long long HW = (long long)vw.W * vw.H;
    const long long p = (long long)pm.py * vw.W + pm.px;
    image[3 * vw.pix_base + p] = C0;
    image[3 * vw.pix_base + HW + p] = C1;
    image[3 * vw.pix_base + 2 * HW + p] = C2;
    alpha[vw.pix_base + p] = 1.f - T;
    depth[vw.pix_base + p] = D;
    B->pix_T[vw.pix_base + p] = T;
    B->pix_last[vw.pix_base + p] = last;
    B->pix_nfrag[vw.pix_base + p] = nfrag;
  }
}

// ---------------------------------------------------------------------------
// K7: backward blend.  Re-walks each tile's list back to front from the last
// blended entry, recomputing every fragment bit for bit, and accumulates the
// gradient of the record fields (warp-reduced, one vector atomic per field
// group and warp) into the per-slot record gradient buffer.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_blend_bwd(const Batch* __restrict__ B,
                                                           const float* __restrict__ dimage,
                                                           const float* __restrict__ dalpha,
                                                           const float* __restrict__ ddepth) {
  constexpr int NT = TILE * TILE;
  __shared__ float4 sm[REC_Q][BLEND_BATCH];
  __shared__ unsigned sslot[BLEND_BATCH];
  __shared__ int smax;
  const int gt = blockIdx.x;
  const ViewD& vw = B->vw[find_view(B, gt)];
  const int lt = gt - vw.tile_base;
  const int tyi = lt / vw.tiles_x, txi = lt - tyi * vw.tiles_x;
  const PixelMap<TILE> pm(txi, tyi);
  const bool inimg = (pm.px < vw.W) & (pm.py < vw.H);
  const float fpx = (float)pm.px + 0.5f, fpy = (float)pm.py + 0.5f;
  const Counters* c = B->ctr;
  const int2 rg = B->ranges[gt];
  const unsigned* __restrict__ vals = B->vals[c->n_passes & 1];
  const float4* __restrict__ rec = B->rec;
  float4* __restrict__ rgrad = B->rec_grad;
  const bool pure = (B->flags & TTS_FLAG_PURE) != 0;
  const float cap = B->alpha_cap, skip = B->alpha_skip;
  const long long HW = (long long)vw.W * vw.H;
  const long long p = (long long)pm.py * vw.W + pm.px;
  float Tfin = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gO = 0.f, gD = 0.f;
  int last = 0;
  if (inimg) {
    Tfin = B->pix_T[vw.pix_base + p];
    last = B->pix_last[vw.pix_base + p];
    gC0 = dimage[3 * vw.pix_base + p];
    gC1 = dimage[3 * vw.pix_base + HW + p];
    gC2 = dimage[3 * vw.pix_base + 2 * HW + p];
    if (dalpha) gO = dalpha[vw.pix_base + p];
    if (ddepth) gD = ddepth[vw.pix_base + p];
  }
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  if (last > 0) atomicMax(&smax, last);
  __syncthreads();
  const int maxlast = smax;
  float T = Tfin, S = 0.f;
  const float gOT = gO * Tfin;
  const int lane = threadIdx.x & 31;
  for (int top = rg.x + maxlast; top > rg.x; top -= BLEND_BATCH) {
    const int base = max(rg.x, top - BLEND_BATCH);
    const int n = top - base;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += NT) {
      const unsigned slot = vals[base + i];
      sslot[i] = slot;
      const float4* r = rec + (size_t)slot * REC_Q;
#pragma unroll
      for (int q = 0; q < REC_Q; ++q) sm[q][i] = __ldg(r + q);
    }
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
      const bool active = (base + j - rg.x) < last;
      const float4 q0 = sm[0][j];
      if (pm.warp_misses(q0)) continue;
      if (!__any_sync(0xffffffffu, active)) continue;
      const Chord ch = chord_eval(q0, sm[1][j], sm[2][j], sm[3][j], fpx, fpy);
      bool contrib = active & ch.hit;
      Opacity o;
      float a = 0.f;
      if (contrib) {
        o = opacity_eval(sm[4][j], ch);
        a = pure ? o.alpha : fminf(o.alpha, cap);
        contrib = pure ? (a > 0.f) : (a >= skip);
      }
      float gP[4] = {0.f, 0.f, 0.f, 0.f}, gA[4] = {0.f, 0.f, 0.f, 0.f}, gB[4] = {0.f, 0.f, 0.f, 0.f};
      float gF = 0.f, gK0 = 0.f, gKx = 0.f, gKy = 0.f, gz = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
      if (contrib) {
        const float4 q5 = sm[5][j];
        const float om = __fsub_rn(1.f, a);
        const float Ti = __fdiv_rn(T, om);
        const float wv = gC0 * q5.y + gC1 * q5.z + gC2 * q5.w + gD * q5.x;
        const float dLda = Ti * wv - (S - gOT) / om;
        S += Ti * a * wv;
        T = Ti;
        const float wgt = Ti * a;
        gz = wgt * gD;
        gc0 = wgt * gC0;
        gc1 = wgt * gC1;
        gc2 = wgt * gC2;
        const bool clamped = !pure && (o.alpha > cap);
        if (!clamped) {
          // alpha = (1 - e1) B with x = s (f_prev - f_next), y = s f_next
          const float dx = dLda * o.e1 * o.B;
          const float dy = -dLda * o.alpha * (1.f - o.B);
          const float iin = o.rho_out * o.r, iout = o.rho_in * o.r;
          const float dpin = -dx * o.sGz * iin * iin;
          const float dpout = (dx - dy) * o.sGz * iout * iout;
          const float dsGz = dx * (ch.p_out - ch.p_in) * o.r - dy * ch.p_out * iout;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float dp = (k == ch.kin) ? dpin : ((k == ch.kout) ? dpout : 0.f);
            gP[k] = dp;
            gA[k] = dp * ch.dx;
            gB[k] = dp * ch.dy;
          }
          gF = dy;
          gK0 = dsGz;
          gKx = (dy + dsGz) * ch.dx;
          gKy = (dy + dsGz) * ch.dy;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, contrib);
      if (m == 0u) continue;
      float4* dst = rgrad + (size_t)sslot[j] * REC_Q;
      if (__popc(m) == 1) {
        if (contrib) {
          atomicAdd(dst + 1, make_float4(gP[0], gP[1], gP[2], gP[3]));
          atomicAdd(dst + 2, make_float4(gA[0], gA[1], gA[2], gA[3]));
          atomicAdd(dst + 3, make_float4(gB[0], gB[1], gB[2], gB[3]));
          atomicAdd(dst + 4, make_float4(gF, gK0, gKx, gKy));
          atomicAdd(dst + 5, make_float4(gz, gc0, gc1, gc2));
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          gP[k] = warp_sum(gP[k]);
          gA[k] = warp_sum(gA[k]);
          gB[k] = warp_sum(gB[k]);
        }
        gF = warp_sum(gF); gK0 = warp_sum(gK0); gKx = warp_sum(gKx); gKy = warp_sum(gKy);
        gz = warp_sum(gz); gc0 = warp_sum(gc0); gc1 = warp_sum(gc1); gc2 = warp_sum(gc2);
        if (lane == 0) {
          atomicAdd(dst + 1, make_float4(gP[0], gP[1], gP[2], gP[3]));
          atomicAdd(dst + 2, make_float4(gA[0], gA[1], gA[2], gA[3]));
          atomicAdd(dst + 3, make_float4(gB[0], gB[1], gB[2], gB[3]));
          atomicAdd(dst + 4, make_float4(gF, gK0, gKx, gKy));
          atomicAdd(dst + 5, make_float4(gz, gc0, gc1, gc2));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K8: record -> vertex adjoint.  One thread per survivor of a scene; loops
// over the scene's views, recomputes the view's tet geometry, applies the
// adjoint of the record fields (App. A.3's affine SDF and the face planes),
// clears the record gradient slot, and scatters into dV, df, drgb.
// The reference point x_r (ray through the bbox corner pixel at the centroid
// depth) is held constant: the fragment opacity does not depend on it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tet_bwd(const Batch* __restrict__ B, GradOut go) {
  const int s = blockIdx.y;
  const SceneD& S = B->sc[s];
  const int nsurv = B->ctr->n_surv[s];
  const float sv = B->s;
  float* __restrict__ gV = go.dV[s];
  float* __restrict__ gf = go.df[s];
  float* __restrict__ gc = go.drgb[s];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nsurv; k += gridDim.x * blockDim.x) {
    const int tet = B->surv[S.surv_off + k];
    TetIn in;
    bool loaded = false;
    float3 dv[4] = {f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0), f3(0, 0, 0)};
    float dfv[4] = {0.f, 0.f, 0.f, 0.f};
    float3 dcol = f3(0, 0, 0);
    bool any = false;
    for (int vi = 0; vi < S.view_cnt; ++vi) {
      const int v = B->scene_views[S.view_off + vi];
      const ViewD& vw = B->vw[v];
      const long long slot = vw.rec_base + k;
      if (B->rec_nt[slot] == 0) continue;
      float4* gq = B->rec_grad + slot * REC_Q;
      const float4 g1 = gq[1], g2 = gq[2], g3 = gq[3], g4 = gq[4], g5 = gq[5];
      const float mag = fabsf(g1.x) + fabsf(g1.y) + fabsf(g1.z) + fabsf(g1.w) + fabsf(g2.x) +
                        fabsf(g2.y) + fabsf(g2.z) + fabsf(g2.w) + fabsf(g3.x) + fabsf(g3.y) +
                        fabsf(g3.z) + fabsf(g3.w) + fabsf(g4.x) + fabsf(g4.y) + fabsf(g4.z) +
                        fabsf(g4.w) + fabsf(g5.x) + fabsf(g5.y) + fabsf(g5.z) + fabsf(g5.w);
      if (mag == 0.f) continue;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      gq[1] = z4; gq[2] = z4; gq[3] = z4; gq[4] = z4; gq[5] = z4;
      if (!loaded) { load_tet(S, tet, in); loaded = true; }
      Geo G;
      tet_geometry(vw, sv, in, G);
      if (!G.visible) continue;
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
      for (int sl = 0; sl < 4; ++sl) {
        const int fk = G.slot_face[sl];
        const int i = kFaceVerts[fk][0], j = kFaceVerts[fk][1], l = kFaceVerts[fk][2];
        const float3 dm = f3(gPs[sl] * xr.x + gAs[sl] * G.zr, gPs[sl] * xr.y + gBs[sl] * G.zr,
                             gPs[sl] * xr.z);
        const float e = G.e[fk];
        const float3 n = G.n[fk];
        const float lam = dot3(n, dm) / (e * e);
        const float3 Xi = G.xm + G.y[i];
        const float3 dn = (1.f / e) * dm - lam * Xi;
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
      const float idet = 1.f / G.det;
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
    }
    if (!any) continue;
    const int4 t = __ldg(&S.T[tet]);
    const int id[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      atomicAdd(gV + 3ll * id[q], dv[q].x);
      atomicAdd(gV + 3ll * id[q] + 1, dv[q].y);
      atomicAdd(gV + 3ll * id[q] + 2, dv[q].z);
      atomicAdd(gf + id[q], dfv[q]);
      atomicAdd(gc + 3ll * id[q], dcol.x);
      atomicAdd(gc + 3ll * id[q] + 1, dcol.y);
      atomicAdd(gc + 3ll * id[q] + 2, dcol.z);
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_blend_fwd(const HostPlan& P, const Batch* dB, float* image, float* alpha, float* depth,
                     cudaStream_t st) {
  switch (P.tile) {
    case 8: k_blend_fwd<8><<<P.total_tiles, 64, 0, st>>>(dB, image, alpha, depth); break;
    case 16: k_blend_fwd<16><<<P.total_tiles, 256, 0, st>>>(dB, image, alpha, depth); break;
    default: k_blend_fwd<32><<<P.total_tiles, 1024, 0, st>>>(dB, image, alpha, depth); break;
  }
  return 1;
}

int launch_blend_bwd(const HostPlan& P, const Batch* dB, const float* dimage, const float* dalpha,
                     const float* ddepth, cudaStream_t st) {
  switch (P.tile) {
    case 8: k_blend_bwd<8><<<P.total_tiles, 64, 0, st>>>(dB, dimage, dalpha, ddepth); break;
    case 16: k_blend_bwd<16><<<P.total_tiles, 256, 0, st>>>(dB, dimage, dalpha, ddepth); break;
    default: k_blend_bwd<32><<<P.total_tiles, 1024, 0, st>>>(dB, dimage, dalpha, ddepth); break;
  }
  return 1;
}

int launch_tet_bwd(const HostPlan& P, const Batch* dB, const GradOut& go, cudaStream_t st) {
  dim3 g(P.tet_bwd_blocks, P.n_scenes);
  k_tet_bwd<<<g, 256, 0, st>>>(dB, go);
  return 1;
}

}  // namespace tts
