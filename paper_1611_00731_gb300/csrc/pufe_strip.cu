// Enrichment strip of H and S on the CUDA cores (mixed path, n_e <= 128).
//
// With the element basis split into the 64 tricubic functions phi_i (F) and
// the enrichments b_r = phi_v^PU Psi_alpha (E), the element integrals of
// Sec. 4 (eq. disceig3d) on the element's shared rule (Sec. 5.2) are
//   H_ir = sum_q w_q [1/2 grad phi_i . grad b_r + V_q phi_i b_r],
//   S_ir = sum_q w_q phi_i b_r,
// for i in F or E and r in E; the FE-FE block is done elsewhere.
//
// F x E block: for fixed r the sum over q is the projection of per-point
// fields onto the tensor-product functions L_a(x) L_b(y) L_c(z), so on a
// p^3 (sub)cell it contracts one axis at a time (sum factorization):
//   f^d = w (d b_r / d x_d) / h_d  (paired with L' along axis d),
//   f^V = w V b_r,  f^S = w b_r,
//   z: X_c = sum L_c f^x, Y_c = sum L_c f^y, Z_c = sum (L'_c f^z + L_c f^V),
//      S_c = sum L_c f^S                       (16 p^3 multiply-adds per r)
//   y: X_bc = sum L_b X_c, W_bc = sum (L'_b Y_c + L_b Z_c), S_bc = sum L_b S_c
//   x: H_abc = sum (L'_a X_bc + L_a W_bc),     S_abc = sum L_a S_bc
// against 5 * 64 p^3 for the direct product.
//
// E x E block: a small dense product over the element's points, symmetric in
// (r, s), so only 4 x 4 tiles with r-block <= s-block are formed:
//   H_rs = sum_q [sum_d y_dr y_ds + V_q z_r z_s],  S_rs = sum_q z_r z_s,
//   y_dr = sqrt(w/2) d b_r / d x_d,  z_r = sqrt(w) b_r.
//
// Every product is an FP32 fused multiply-add with round to nearest; the
// element block is added into the FP64 CSR values with atomics (both
// triangles, through the element's scatter map).
#include <algorithm>

#include "pufe_internal.h"

namespace pufe {
namespace {

constexpr int ST_NT = 256;
constexpr int ST_KC = 32;   // points per E x E chunk

__device__ __forceinline__ void lag3vd(float t, float *L, float *dL) {
  const float a = t + 1.0f, b = t + (1.0f / 3.0f), c = t - (1.0f / 3.0f), d = t - 1.0f;
  L[0] = -0.5625f * b * c * d;
  L[1] = 1.6875f * a * c * d;
  L[2] = -1.6875f * a * b * d;
  L[3] = 0.5625f * a * b * c;
  dL[0] = -0.5625f * (c * d + b * d + b * c);
  dL[1] = 1.6875f * (c * d + a * d + a * c);
  dL[2] = -1.6875f * (b * d + a * d + a * b);
  dL[3] = 0.5625f * (b * c + a * c + a * b);
}

// b_r and its physical gradient at one point
struct EnrVal {
  float b, bx, by, bz;
};

// floor(x / d) for 0 <= x <= 2^16 and 1 <= d < 2^16: the high word of
// x * ceil(2^32 / d) (one __umulhi); the rounding error is below
// x 2^-32 <= 2^-16 < 1/d, so it cannot carry the quotient past the next
// integer.  d = 1 (multiplier 2^32) is taken apart.
struct FastDiv {
  unsigned m;
  bool one;
  __device__ explicit FastDiv(int d)
      : m(d > 1 ? (unsigned)((0x100000000ull + (unsigned)d - 1) / (unsigned)d) : 0u), one(d <= 1) {}
  __device__ __forceinline__ int div(int x) const {
    return one ? x : (int)__umulhi((unsigned)x, m);
  }
};

// per-element state shared by the (sub)cell passes
struct StripElem {
  int n, ne, ne8, A, qs, p;
  int64_t q0;
  const int32_t *m;
  const float *pe;
  const float4 *qe;
  const double *V;
  bool wantH, wantS, useV;
  float sx, sy, sz;
  // shared memory
  float *stage, *work, *HE, *SE, *L1, *D1;
  const int *ecs;
  int pm, wfloats;
  // E x E tile of this thread
  int rb, sb, pg, PG;
  bool act;
};

// one (sub)cell of p^3 points starting at element point qs; STAGED: its Psi
// rows ([slot][comp][point], pitch P), points and V are in shared memory
template <bool STAGED>
__device__ __forceinline__ void strip_part(const StripElem &E, double *__restrict__ H,
                                           double *__restrict__ S) {
  const int tid = threadIdx.x;
  const int p = E.p, p2 = p * p, p3 = p2 * p, qs = E.qs, ne = E.ne, ne8 = E.ne8, A = E.A;
  const int P = p3 | 1;
  const float4 *xd = reinterpret_cast<const float4 *>(E.stage + ((A * 4 * P + 3) & ~3));
  const float *vd = reinterpret_cast<const float *>(xd + p3);
  // lq: point index within the (sub)cell
  auto psv = [&](int lq, int slot, int comp) -> float {
    if (STAGED) return E.stage[(slot * 4 + comp) * P + lq];
    const int ql = qs + lq;
    return E.pe[((int64_t)(ql >> 3) * A + slot) * 32 + comp * 8 + (ql & 7)];
  };
  auto xval = [&](int lq) -> float4 { return STAGED ? xd[lq] : E.qe[qs + lq]; };
  auto vval = [&](int lq) -> float {
    if (STAGED) return vd[lq];
    return E.useV ? (float)E.V[E.q0 + qs + lq] : 0.0f;
  };
  auto enr = [&](int lq, int code, float4 x4) -> EnrVal {
    const int lv = code & 7, slot = code >> 3;
    const float fx = (lv & 1) ? 1.0f + x4.x : 1.0f - x4.x;
    const float fy = (lv & 2) ? 1.0f + x4.y : 1.0f - x4.y;
    const float fz = (lv & 4) ? 1.0f + x4.z : 1.0f - x4.z;
    const float gx = (lv & 1) ? 0.125f * E.sx : -0.125f * E.sx;
    const float gy = (lv & 2) ? 0.125f * E.sy : -0.125f * E.sy;
    const float gz = (lv & 4) ? 0.125f * E.sz : -0.125f * E.sz;
    const float phi = 0.125f * fx * fy * fz;
    const float p0 = psv(lq, slot, 0), p1 = psv(lq, slot, 1), p2v = psv(lq, slot, 2),
                p3v = psv(lq, slot, 3);
    EnrVal o;
    o.b = phi * p0;
    o.bx = fmaf(gx * fy * fz, p0, phi * p1);
    o.by = fmaf(fx * gy * fz, p0, phi * p2v);
    o.bz = fmaf(fx * fy * gz, p0, phi * p3v);
    return o;
  };
  const float ihx = 0.5f * E.sx, ihy = 0.5f * E.sy, ihz = 0.5f * E.sz;   // 1 / h_d
  const int pm = E.pm;
  const float *L1 = E.L1, *D1 = E.D1;
  const int32_t *m = E.m;
  const int n = E.n;

  // ---- F x E block ---------------------------------------------------------
  const int per_r = p2 * 20 + p * 48;
  const int G = max(1, min(min(ne, E.wfloats / per_r), ST_NT / p2));
  const FastDiv dp2(p2), dp16(p * 16);
  for (int r0 = 0; r0 < ne; r0 += G) {
    const int Gc = min(G, ne - r0);
    float *T1 = E.work;                   // [Gc][p^2][20]: X, Y, Z, S (x4), pad
    float *T2 = E.work + Gc * p2 * 20;    // [Gc][p][16][3]
    __syncthreads();
    // z: one thread per (r, qx, qy) column
    for (int it = tid; it < Gc * p2; it += ST_NT) {
      const int g = dp2.div(it), qxy = it - g * p2;
      const int code = E.ecs[r0 + g];
      float X[4] = {0.f, 0.f, 0.f, 0.f}, Y[4] = {0.f, 0.f, 0.f, 0.f};
      float Z[4] = {0.f, 0.f, 0.f, 0.f}, Sa[4] = {0.f, 0.f, 0.f, 0.f};
      for (int qz = 0; qz < p; ++qz) {
        const int lq = qxy + p2 * qz;
        const float4 x4 = xval(lq);
        const float vq = vval(lq);
        const EnrVal ev = enr(lq, code, x4);
        const float fx = x4.w * ev.bx * ihx, fy = x4.w * ev.by * ihy, fz = x4.w * ev.bz * ihz;
        const float fS = x4.w * ev.b, fV = fS * vq;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float Lc = L1[(8 + c) * pm + qz], Dc = D1[(8 + c) * pm + qz];
          X[c] = fmaf(Lc, fx, X[c]);
          Y[c] = fmaf(Lc, fy, Y[c]);
          Z[c] = fmaf(Dc, fz, fmaf(Lc, fV, Z[c]));
          Sa[c] = fmaf(Lc, fS, Sa[c]);
        }
      }
      float4 *t1 = reinterpret_cast<float4 *>(T1 + (size_t)it * 20);
      t1[0] = make_float4(X[0], X[1], X[2], X[3]);
      t1[1] = make_float4(Y[0], Y[1], Y[2], Y[3]);
      t1[2] = make_float4(Z[0], Z[1], Z[2], Z[3]);
      t1[3] = make_float4(Sa[0], Sa[1], Sa[2], Sa[3]);
    }
    __syncthreads();
    // y: one thread per (r, qx, b, c)
    for (int it = tid; it < Gc * p * 16; it += ST_NT) {
      const int g = dp16.div(it), rem = it - g * p * 16;
      const int qx = rem >> 4, bc = rem & 15, b = bc >> 2, c = bc & 3;
      float x2 = 0.0f, w2 = 0.0f, s2 = 0.0f;
      const float *t1 = T1 + (size_t)(g * p2 + qx) * 20;
      for (int qy = 0; qy < p; ++qy, t1 += p * 20) {
        const float Lb = L1[(4 + b) * pm + qy], Db = D1[(4 + b) * pm + qy];
        x2 = fmaf(Lb, t1[c], x2);
        w2 = fmaf(Db, t1[4 + c], fmaf(Lb, t1[8 + c], w2));
        s2 = fmaf(Lb, t1[12 + c], s2);
      }
      float *t2 = T2 + (size_t)it * 3;
      t2[0] = x2;
      t2[1] = w2;
      t2[2] = s2;
    }
    __syncthreads();
    // x: one thread per (r, i), i = a + 4b + 16c; add into both triangles
    for (int it = tid; it < Gc * 64; it += ST_NT) {
      const int g = it >> 6, i = it & 63, r = r0 + g;
      const int a = i & 3, bc = ((i >> 2) & 3) * 4 + (i >> 4);
      float hs = 0.0f, ss = 0.0f;
      const float *t2 = T2 + ((size_t)g * p * 16 + bc) * 3;
      for (int qx = 0; qx < p; ++qx, t2 += 48) {
        hs = fmaf(D1[a * pm + qx], t2[0], fmaf(L1[a * pm + qx], t2[1], hs));
        ss = fmaf(L1[a * pm + qx], t2[2], ss);
      }
      const int s_ir = m[i * n + 64 + r], s_ri = m[(64 + r) * n + i];
      if (E.wantH) {
        atomicAdd(H + s_ir, (double)hs);
        atomicAdd(H + s_ri, (double)hs);
      }
      if (E.wantS) {
        atomicAdd(S + s_ir, (double)ss);
        atomicAdd(S + s_ri, (double)ss);
      }
    }
  }

  // ---- E x E block over this (sub)cell's points --------------------------------
  float h16[16], s16[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) h16[u] = s16[u] = 0.0f;
  const int ld = 4 * ne8;   // floats per point in the chunk table
  float *Xt = E.work;       // [ST_KC][4][ne8]: y_0, y_1, y_2, z
  float *Vc = E.work + ST_KC * ld;
  const FastDiv dne8(ne8);
  for (int c0 = 0; c0 < p3; c0 += ST_KC) {
    __syncthreads();
    for (int it = tid; it < ST_KC * ne8; it += ST_NT) {
      const int qq = dne8.div(it), r = it - qq * ne8;
      float y0 = 0.f, y1 = 0.f, y2 = 0.f, z = 0.f;
      if (c0 + qq < p3 && r < ne) {
        const int lq = c0 + qq;
        const float4 x4 = xval(lq);
        const EnrVal ev = enr(lq, E.ecs[r], x4);
        const float shalf = sqrtf(0.5f * x4.w), sw = sqrtf(x4.w);
        y0 = shalf * ev.bx;
        y1 = shalf * ev.by;
        y2 = shalf * ev.bz;
        z = sw * ev.b;
      }
      float *xr = Xt + qq * ld + r;
      xr[0] = y0;
      xr[ne8] = y1;
      xr[2 * ne8] = y2;
      xr[3 * ne8] = z;
    }
    if (tid < ST_KC) Vc[tid] = (c0 + tid < p3) ? vval(c0 + tid) : 0.0f;
    __syncthreads();
    if (E.act) {
      const int qend = min(ST_KC, p3 - c0);
      for (int qq = E.pg; qq < qend; qq += E.PG) {
        const float *xq = Xt + qq * ld;
        float4 ar[4], as[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          ar[kk] = *reinterpret_cast<const float4 *>(xq + kk * ne8 + 4 * E.rb);
          as[kk] = *reinterpret_cast<const float4 *>(xq + kk * ne8 + 4 * E.sb);
        }
        const float v = Vc[qq];
        const float r0v[4] = {ar[0].x, ar[0].y, ar[0].z, ar[0].w};
        const float r1v[4] = {ar[1].x, ar[1].y, ar[1].z, ar[1].w};
        const float r2v[4] = {ar[2].x, ar[2].y, ar[2].z, ar[2].w};
        const float r3v[4] = {ar[3].x, ar[3].y, ar[3].z, ar[3].w};
        const float s0v[4] = {as[0].x, as[0].y, as[0].z, as[0].w};
        const float s1v[4] = {as[1].x, as[1].y, as[1].z, as[1].w};
        const float s2v[4] = {as[2].x, as[2].y, as[2].z, as[2].w};
        const float s3v[4] = {as[3].x, as[3].y, as[3].z, as[3].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float rv = v * r3v[i];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float h = h16[i * 4 + j];
            h = fmaf(r0v[i], s0v[j], h);
            h = fmaf(r1v[i], s1v[j], h);
            h = fmaf(r2v[i], s2v[j], h);
            h16[i * 4 + j] = fmaf(rv, s3v[j], h);
            s16[i * 4 + j] = fmaf(r3v[i], s3v[j], s16[i * 4 + j]);
          }
        }
      }
    }
  }
  if (E.act) {   // the PG point groups meet in shared memory
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        atomicAdd(&E.HE[(4 * E.rb + i) * ne8 + 4 * E.sb + j], h16[i * 4 + j]);
        atomicAdd(&E.SE[(4 * E.rb + i) * ne8 + 4 * E.sb + j], s16[i * 4 + j]);
      }
  }
}

__global__ void __launch_bounds__(ST_NT, 2) k_strip_sf(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const double *__restrict__ V, const int32_t *__restrict__ partoff,
    const int32_t *__restrict__ part_p, const int32_t *__restrict__ part_q,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ ecol,
    const int32_t *__restrict__ aoff, const int64_t *__restrict__ toff32,
    const float *__restrict__ psi, const int64_t *__restrict__ soff,
    const int32_t *__restrict__ smap, float sx, float sy, float sz, int pm, int wfloats,
    int sfloats, int what, double *__restrict__ H, double *__restrict__ S, unsigned *err) {
  extern __shared__ float4 sm_st4[];
  const int e = order[blockIdx.x], tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  StripElem E;
  E.n = (int)(doff[e + 1] - doff[e]);
  E.ne = E.n - 64;
  if (E.ne <= 0) return;   // FE-only element: no strip
  if (E.n > 128) {
    if (tid == 0) atomicOr(err, DEVERR_SHAPE);
    return;
  }
  const int ne = E.ne, ne8 = (ne + 7) & ~7;
  E.ne8 = ne8;
  E.q0 = qoff[e];
  E.A = aoff[e + 1] - aoff[e];
  E.m = smap + soff[e];
  E.pe = psi + 4 * toff32[e];
  E.qe = qdat + qpoff[e];
  E.V = V;
  E.wantH = (what & PUFE_WANT_H) != 0;
  E.wantS = (what & PUFE_WANT_S) != 0;
  E.useV = E.wantH && V != nullptr;
  E.sx = sx;
  E.sy = sy;
  E.sz = sz;
  E.pm = pm;
  E.wfloats = wfloats;

  // shared memory: [stage: sfloats][work: wfloats][HE, SE: ne8^2 each]
  //                [L1, D1: 12 pm each][ecs: ne]
  E.stage = reinterpret_cast<float *>(sm_st4);
  E.work = E.stage + sfloats;
  E.HE = E.work + wfloats;   // [ne8][ne8], entries r <= s
  E.SE = E.HE + ne8 * ne8;
  E.L1 = E.SE + ne8 * ne8;   // [3][4][pm]
  E.D1 = E.L1 + 12 * pm;     // [3][4][pm]
  int *ecs = reinterpret_cast<int *>(E.D1 + 12 * pm);
  E.ecs = ecs;
  if (tid < ne) ecs[tid] = ecol[(doff[e] - 64ll * e) + tid];
  for (int o = tid; o < 2 * ne8 * ne8; o += ST_NT) E.HE[o] = 0.0f;

  // E x E tiles: 4 x 4 blocks (rb <= sb), one per lane; WG warps cover the
  // tiles, the PG = 8 / WG warp groups split the points, so the lanes of a
  // warp read the same point (broadcast-friendly shared-memory reads)
  const int nb = ne8 >> 2, ntile = nb * (nb + 1) / 2;
  const int WG = ntile <= 32 ? 1 : (ntile <= 64 ? 2 : (ntile <= 128 ? 4 : 8));
  E.PG = (ST_NT / 32) / WG;
  const int tile = (warp % WG) * 32 + lane;
  E.pg = warp / WG;
  E.act = tile < ntile;
  int rb = 0, tt = E.act ? tile : 0;
  while (tt >= nb - rb) {
    tt -= nb - rb;
    ++rb;
  }
  E.rb = rb;
  E.sb = rb + tt;

  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    const int p = part_p[k];
    const int p2 = p * p, p3 = p2 * p;
    if (p > pm || p2 * 20 + p * 48 > wfloats || ST_KC * (4 * ne8 + 1) > wfloats) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    E.p = p;
    E.qs = part_q[k];
    const int P = p3 | 1, A = E.A, qs = E.qs;
    const bool staged = ((A * 4 * P + 3) & ~3) + 5 * p3 <= sfloats;
    __syncthreads();   // previous users of stage/work/L1/D1 are done
    if (staged) {   // Psi transposed to [slot][comp][point], pitch P (odd)
      float *stage = E.stage;
      float4 *xd = reinterpret_cast<float4 *>(stage + ((A * 4 * P + 3) & ~3));
      float *vd = reinterpret_cast<float *>(xd + p3);
      const int blk0 = qs >> 3, nblk = ((qs + p3 + 7) >> 3) - blk0;
      const float4 *src = reinterpret_cast<const float4 *>(E.pe + (int64_t)blk0 * A * 32);
      const FastDiv dA8(A * 8);
      for (int o = tid; o < nblk * A * 8; o += ST_NT) {   // one float4 = 4 points of a row
        const float4 v4 = src[o];
        const int blk = dA8.div(o), rem = o - blk * (A * 8);
        const int row = rem >> 1;   // slot * 4 + comp
        const int qb = (blk0 + blk) * 8 + (rem & 1) * 4 - qs;
        float *d = stage + row * P;
        if (qb >= 0 && qb < p3) d[qb] = v4.x;
        if (qb + 1 >= 0 && qb + 1 < p3) d[qb + 1] = v4.y;
        if (qb + 2 >= 0 && qb + 2 < p3) d[qb + 2] = v4.z;
        if (qb + 3 >= 0 && qb + 3 < p3) d[qb + 3] = v4.w;
      }
      for (int o = tid; o < p3; o += ST_NT) {
        xd[o] = E.qe[qs + o];
        vd[o] = E.useV ? (float)V[E.q0 + qs + o] : 0.0f;
      }
    }
    for (int o = tid; o < 3 * p; o += ST_NT) {
      const int d = o / p, t = o - d * p;
      const int stride = d == 0 ? 1 : (d == 1 ? p : p2);
      const float4 x4 = E.qe[qs + t * stride];
      float L[4], dL[4];
      lag3vd(d == 0 ? x4.x : (d == 1 ? x4.y : x4.z), L, dL);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        E.L1[(d * 4 + a) * pm + t] = L[a];
        E.D1[(d * 4 + a) * pm + t] = dL[a];
      }
    }
    if (staged)
      strip_part<true>(E, H, S);
    else
      strip_part<false>(E, H, S);
  }
  __syncthreads();
  // ---- E x E into the FP64 CSR values, both triangles ---------------------------
  const FastDiv dne(ne);
  for (int o = tid; o < ne * ne; o += ST_NT) {
    const int r = dne.div(o), sc = o - r * ne;
    const int lo = min(r, sc), hi = max(r, sc);
    const int slot = E.m[(64 + r) * E.n + 64 + sc];
    if (E.wantH) atomicAdd(H + slot, (double)E.HE[lo * ne8 + hi]);
    if (E.wantS) atomicAdd(S + slot, (double)E.SE[lo * ne8 + hi]);
  }
}

}  // namespace

// Shared-memory floats of the strip kernel's work area: the F x E
// intermediates of one group of enrichments (as many as keep 256 threads
// busy, at least 1) for every per-axis count in `pmask`, or one E x E chunk
// table for enrichment count (rounded to 8) ne8.
static int strip_work_floats(uint32_t pmask, int ne8) {
  int w = ST_KC * (4 * ne8 + 1);
  for (int p = 1; p < 32; ++p) {
    if (!(pmask & (1u << p))) continue;
    const int per_r = p * p * 20 + p * 48;
    const int g = std::max(1, std::min(ne8, ST_NT / (p * p)));
    w = std::max(w, g * per_r);
  }
  return (w + 3) & ~3;
}

pufe_status launch_strip_sf(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                            int first, int count, cudaStream_t st) {
  if (count <= 0) return PUFE_OK;
  auto &D = ctx->d;
  int ne8 = 8;
  for (int64_t k = first; k < first + count; ++k)
    ne8 = std::max(ne8, (ctx->n_e[ctx->order[k]] - 64 + 7) & ~7);
  const int sneed = ctx->strip_stage;
  if (ne8 > 64) return fail(PUFE_EINVAL, "strip kernel takes n_e <= 128");
  const int pm = std::max(1, ctx->max_part_p);
  const int wf = strip_work_floats(ctx->strip_pmask, ne8);
  const int sf = (sneed + 3) & ~3;
  const size_t sm = ((size_t)sf + wf + 2 * ne8 * ne8 + 24 * pm + ne8) * sizeof(float);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "strip kernel: shared memory above 227 KB");
  PUFE_CUDA_TRY(cudaFuncSetAttribute(k_strip_sf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_strip_sf<<<(unsigned)count, ST_NT, sm, st>>>(
      D.order + first, D.qoff, D.qpoff, D.qdat, V, D.partoff, D.part_p, D.part_q, D.doff, D.ecol,
      D.aoff, D.toff32, D.psi32, D.soff, D.smap, (float)(2.0 / ctx->h[0]),
      (float)(2.0 / ctx->h[1]), (float)(2.0 / ctx->h[2]), pm, wf, sf, what, H, S, D.err);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

}  // namespace pufe

