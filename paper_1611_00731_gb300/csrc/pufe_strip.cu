// Enrichment strip of H and S on the CUDA cores (mixed path, n_e <= 128).
//
// With the element basis split into the 64 tricubic functions phi_i (F) and
// the enrichments b_r = phi_v^PU Psi_alpha (E), the element integrals of
// Sec. 4 (eq. disceig3d) on the element's shared rule (Sec. 5.2) are
//   H_ir = sum_q w_q [1/2 grad phi_i . grad b_r + V_q phi_i b_r],
//   S_ir = sum_q w_q phi_i b_r,
// for i in F or E and r in E; the FE-FE block is done elsewhere.
//
// F x E block, slot form: the trilinear PU factor of r = (v, alpha) is a
// product of linears 1 -+ xi per axis, so all eight vertex columns of a slot
// alpha are projections of the slot's four per-point fields (w Psi,
// w V Psi, w grad Psi) onto tensor products of L_a (1 -+ xi), L'_a (1 -+ xi)
// and L'_a along each axis, contracted one axis at a time on a p^3
// (sub)cell (sum factorization; the expansion is written out in
// strip_part), about 48 p^3 multiply-adds per slot against 5 * 64 * 8 p^3
// for the direct products of its eight columns.
//
// E x E block of H, direct form: a small dense product over the element's
// points, symmetric in (r, s), so only 4 x 4 tiles with r-block <= s-block are
// formed:
//   H_rs = sum_q [sum_d y_dr y_ds + V_q z_r z_s],
//   y_dr = sqrt(w/2) d b_r / d x_d,  z_r = sqrt(w) b_r.
// The E x E block of S is computed with FP64-class sums by its own kernel
// (pufe_see.cu).
//
// E x E block of H, enrichment-pair form: for r = (v, alpha), s = (v', beta) the
// PU factors are trilinear, phi_v = 1/8 prod_d (1 + s_d x_d) with s_d = +-1,
// so along each axis phi_v phi_v' is one of u_0 = (1-x)^2, u_1 = 1 - x^2,
// u_2 = (1+x)^2 (index b_d + b'_d, b = (s + 1) / 2), d phi_v / dx_d is a
// constant and phi_v' is one of l_0 = 1 - x, l_1 = 1 + x.  Expanding
// grad b_r . grad b_s, every entry of the pair's 64 vertex pairs is a signed
// sum of projections of eight per-point fields of (alpha, beta) alone,
//   A = w Psi_a Psi_b,  E = w (V Psi_a Psi_b + 1/2 grad Psi_a . grad Psi_b),
//   B_d = w Psi_b d_d Psi_a,  C_d = w Psi_a d_d Psi_b,
// onto tensor products of {u_k, 1, l_t}:
//   64 H_rs = <E, u u u> + 1/2 sum_d (2/h_d)^2 s_d s'_d <A, u u with 1 on d>
//           + 1/2 sum_d (2/h_d) (s_d <C_d, u u with l_b'd on d>
//                                + s'_d <B_d, u u with l_bd on d>).
// The 189 projections of a pair are contracted axis by axis (z: 23 per
// column, y: 66 per line, x: 189), about 56 p^3 + 200 p^2 operations against
// 5 x 64 p^3 for the direct products of the pair's vertex pairs.  An element
// takes this form when its enrichments have at most 8 slots and the form's
// operation count is below the direct one.
//
// Every product is an FP32 fused multiply-add with round to nearest; the
// element block is added into the FP64 CSR values with atomics (both
// triangles, through the element's scatter map).
#include <algorithm>
#include <cstdlib>
#include <fstream>
#include <map>
#include <string>

#include "pufe_internal.h"

namespace pufe {
namespace {

constexpr int ST_NT = 256;
constexpr int ST_KC = 32;   // points per E x E chunk
// registers per thread: 80 lets three 256-thread CTAs share an SM (when
// their shared memory fits, <= 75 KB each)
constexpr int ST_MAXREG = 80;

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

// floor(x / d) for 0 <= x and 1 <= d with x d < 2^32: the high word of
// x * ceil(2^32 / d) (one __umulhi).  The multiplier exceeds 2^32 / d by less
// than 1, so the product exceeds x 2^32 / d by less than x, i.e. the quotient
// by less than x / 2^32 < 1 / d, which cannot carry it past the next integer
// (the fractional part of x / d is at most 1 - 1/d).  d = 1 (multiplier
// 2^32) is taken apart.  Every use below divides a loop index bounded by the
// launch sizes (p <= 16 points per axis, n_e <= 128, so at most 64
// enrichment columns and slots); strip_launch and the adjoint launcher check
// the largest product x d against 2^32 on the host.
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
  float *stage, *work, *HE;
  // 1D factors of the F x E slot form per axis d and 1D point t:
  // T4[(d pm + t) 2 + l] = (L_a l_l)_a, T4[6 pm + (d pm + t) 2 + l] = (L'_a l_l)_a,
  // T4[12 pm + d pm + t] = (L'_a)_a, T4[15 pm + d pm + t] = (L_a)_a
  // (a = 0..3 in the four components)
  const float4 *T4;
  const int *scol;   // [slot][vertex]: column of (slot, vertex), -1 if absent
  bool fxs;          // F x E block in the slot form (else column by column)
  const int *ecs;
  int pm, wfloats;
  // E x E tile of this thread (direct form)
  int rb, sb, pg, PG;
  bool act;
  // enrichment-pair form: pair list (alpha | beta << 8), projections
  // [pair][189] and the 1D factors [axis][u_0, u_1, u_2, 1, l_0, l_1][pm]
  bool sp;
  int npair;
  const int *pairs;
  float *PE;
  const float *F1;
  // Bloch scatter: lattice-shift code of each column, the 8 phases
  // exp(i k.R) in FP32, imaginary outputs
  const uint8_t *esh;
  const float *phr, *phi;
  double *Hi, *Si;
};

// phase conj(exp(i k.R_a)) exp(i k.R_b) of a column pair with shift codes a, b
__device__ __forceinline__ void pair_phase(const StripElem &E, int a, int b, float &pr, float &pi) {
  pr = E.phr[a] * E.phr[b] + E.phi[a] * E.phi[b];
  pi = E.phr[a] * E.phi[b] - E.phi[a] * E.phr[b];
}

// Row groups of the enrichment-pair contraction.  z-stage outputs (rows a):
// 0-2 A u_k, 3 A, 4-6 E u_k, 7-9 B_x u_k, 10-12 C_x u_k, 13-15 B_y u_k,
// 16-18 C_y u_k, 19-20 B_z l_t, 21-22 C_z l_t.  Factor index f: 0-2 u_k,
// 3 the constant, 4-5 l_t.  Row a of the z stage feeds y outputs j0 .. j0+n-1
// with factors f0 .. f0+n-1, and rows 0-2 also feed j = 9 + a with f = 3:
//   y outputs 0-8 A(u,u), 9-11 A(u,1), 12-14 A(1,u), 15-23 E(u,u),
//   24-32 B_x(u,u), 33-41 C_x(u,u), 42-47 B_y(u,l), 48-53 C_y(u,l),
//   54-59 B_z(l,u), 60-65 C_z(l,u)    (z factor first).
__device__ __forceinline__ void sp_yrow(int a, int &j0, int &f0, int &n) {
  if (a < 3) { j0 = 3 * a; f0 = 0; n = 3; }
  else if (a == 3) { j0 = 12; f0 = 0; n = 3; }
  else if (a < 13) { j0 = 15 + 3 * (a - 4); f0 = 0; n = 3; }
  else if (a < 19) { j0 = 42 + 2 * (a - 13); f0 = 4; n = 2; }
  else { j0 = 54 + 3 * (a - 19); f0 = 0; n = 3; }
}

// Row j of the y stage feeds projections i0 .. i0+n-1 with x factors
// f0 .. f0+n-1, and rows 0-8 also feed i = 27 + j with f = 3; projections:
//   0-26 <A,u u u> (z,y,x), 27-35 <A,u u 1>, 36-44 <A,u 1 u>, 45-53 <A,1 u u>,
//   54-80 <E,u u u>, 81-98 <B_x,u u l>, 99-116 <C_x,u u l>,
//   117-134 <B_y,u l u>, 135-152 <C_y,u l u>, 153-170 <B_z,l u u>, 171-188 <C_z,l u u>
__device__ __forceinline__ void sp_xrow(int j, int &i0, int &f0, int &n) {
  if (j < 9) { i0 = 3 * j; f0 = 0; n = 3; }
  else if (j < 24) { i0 = 36 + 3 * (j - 9); f0 = 0; n = 3; }
  else if (j < 42) { i0 = 81 + 2 * (j - 24); f0 = 4; n = 2; }
  else { i0 = 117 + 3 * (j - 42); f0 = 0; n = 3; }
}

// one (sub)cell of p^3 points starting at element point qs; STAGED: its Psi
// rows ([slot][comp][point], pitch P), points and V are in shared memory
template <bool STAGED, bool BLOCH>
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
  const int pm = E.pm;
  const int32_t *m = E.m;
  const int n = E.n;

  // one (i, r) entry of the F x E block into both triangles of H and S
  auto add_fe = [&](int i, int r, float hs, float ss) {
    const int s_ir = m[i * n + 64 + r], s_ri = m[(64 + r) * n + i];
    if (BLOCH) {   // (i, r) with conj(ph_i) ph_r, (r, i) with its conjugate
      float pr, pi;
      pair_phase(E, E.esh[i], E.esh[64 + r], pr, pi);
      if (E.wantH) {
        atomicAdd(H + s_ir, (double)(hs * pr));
        atomicAdd(E.Hi + s_ir, (double)(hs * pi));
        atomicAdd(H + s_ri, (double)(hs * pr));
        atomicAdd(E.Hi + s_ri, (double)(-hs * pi));
      }
      if (E.wantS) {
        atomicAdd(S + s_ir, (double)(ss * pr));
        atomicAdd(E.Si + s_ir, (double)(ss * pi));
        atomicAdd(S + s_ri, (double)(ss * pr));
        atomicAdd(E.Si + s_ri, (double)(-ss * pi));
      }
    } else {
      if (E.wantH) {
        atomicAdd(H + s_ir, (double)hs);
        atomicAdd(H + s_ri, (double)hs);
      }
      if (E.wantS) {
        atomicAdd(S + s_ir, (double)ss);
        atomicAdd(S + s_ri, (double)ss);
      }
    }
  };
  const float4 *MT = E.T4, *DT = E.T4 + 6 * pm, *D0T = E.T4 + 12 * pm, *LT = E.T4 + 15 * pm;
  const FastDiv dp2(p2), dp(p), dp16(p * 16);

  // ---- F x E block, column form ----------------------------------------------
  // For fixed r the sum over q is the projection of per-point fields onto
  // L_a(x) L_b(y) L_c(z), contracted one axis at a time:
  //   f^d = w (d b_r / d x_d) / h_d  (paired with L' along axis d),
  //   f^V = w V b_r,  f^S = w b_r,
  //   z: X_c = sum L_c f^x, Y_c = sum L_c f^y, Z_c = sum (L'_c f^z + L_c f^V),
  //      S_c = sum L_c f^S                       (16 p^3 multiply-adds per r)
  //   y: X_bc = sum L_b X_c, W_bc = sum (L'_b Y_c + L_b Z_c), S_bc = sum L_b S_c
  //   x: H_abc = sum (L'_a X_bc + L_a W_bc),     S_abc = sum L_a S_bc
  // (b_r evaluated at every point for each column); taken when the element's
  // slots hold few vertex columns each, where the slot form's per-slot y and
  // x stages would cost more.
  if (!E.fxs) {
    const float ihx = 0.5f * E.sx, ihy = 0.5f * E.sy, ihz = 0.5f * E.sz;   // 1 / h_d
    const int per_r = p2 * 20 + p * 48;
    const int G = max(1, min(min(ne, E.wfloats / per_r), ST_NT / p2));
    for (int r0 = 0; r0 < ne; r0 += G) {
      const int Gc = min(G, ne - r0);
      float *T1 = E.work;                   // [Gc][p^2][20]: X, Y, Z, S (x4), pad
      float *T2 = E.work + Gc * p2 * 20;    // [Gc][p][16][3]
      __syncthreads();
      // z: one thread per (r, qx, qy) column
      for (int it = tid; it < Gc * p2; it += ST_NT) {
        const int g = dp2.div(it), qxy = it - g * p2;
        const int code = E.ecs[r0 + g];
        float4 X = make_float4(0.f, 0.f, 0.f, 0.f), Y = X, Z = X, Sa = X;
        for (int qz = 0; qz < p; ++qz) {
          const int lq = qxy + p2 * qz;
          const float4 x4 = xval(lq);
          const float vq = vval(lq);
          const EnrVal ev = enr(lq, code, x4);
          const float fx = x4.w * ev.bx * ihx, fy = x4.w * ev.by * ihy, fz = x4.w * ev.bz * ihz;
          const float fS = x4.w * ev.b, fV = fS * vq;
          const float4 Lc = LT[2 * pm + qz], Dc = D0T[2 * pm + qz];
          X.x = fmaf(Lc.x, fx, X.x);
          X.y = fmaf(Lc.y, fx, X.y);
          X.z = fmaf(Lc.z, fx, X.z);
          X.w = fmaf(Lc.w, fx, X.w);
          Y.x = fmaf(Lc.x, fy, Y.x);
          Y.y = fmaf(Lc.y, fy, Y.y);
          Y.z = fmaf(Lc.z, fy, Y.z);
          Y.w = fmaf(Lc.w, fy, Y.w);
          Z.x = fmaf(Dc.x, fz, fmaf(Lc.x, fV, Z.x));
          Z.y = fmaf(Dc.y, fz, fmaf(Lc.y, fV, Z.y));
          Z.z = fmaf(Dc.z, fz, fmaf(Lc.z, fV, Z.z));
          Z.w = fmaf(Dc.w, fz, fmaf(Lc.w, fV, Z.w));
          Sa.x = fmaf(Lc.x, fS, Sa.x);
          Sa.y = fmaf(Lc.y, fS, Sa.y);
          Sa.z = fmaf(Lc.z, fS, Sa.z);
          Sa.w = fmaf(Lc.w, fS, Sa.w);
        }
        float4 *t1 = reinterpret_cast<float4 *>(T1 + (size_t)it * 20);
        t1[0] = X;
        t1[1] = Y;
        t1[2] = Z;
        t1[3] = Sa;
      }
      __syncthreads();
      // y: one thread per (r, qx, b, c)
      for (int it = tid; it < Gc * p * 16; it += ST_NT) {
        const int g = dp16.div(it), rem = it - g * p * 16;
        const int qx = rem >> 4, bc = rem & 15, b = bc >> 2, c = bc & 3;
        float x2 = 0.0f, w2 = 0.0f, s2 = 0.0f;
        const float *t1 = T1 + (size_t)(g * p2 + qx) * 20;
        const float *lb = reinterpret_cast<const float *>(LT + pm) + b;
        const float *db = reinterpret_cast<const float *>(D0T + pm) + b;
        for (int qy = 0; qy < p; ++qy, t1 += p * 20) {
          const float Lb = lb[4 * qy], Db = db[4 * qy];
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
      // x: one thread per (r, i), i = a + 4b + 16c
      for (int it = tid; it < Gc * 64; it += ST_NT) {
        const int g = it >> 6, i = it & 63, r = r0 + g;
        const int a = i & 3, bc = ((i >> 2) & 3) * 4 + (i >> 4);
        float hs = 0.0f, ss = 0.0f;
        const float *t2 = T2 + ((size_t)g * p * 16 + bc) * 3;
        const float *la = reinterpret_cast<const float *>(LT) + a;
        const float *da = reinterpret_cast<const float *>(D0T) + a;
        for (int qx = 0; qx < p; ++qx, t2 += 48) {
          hs = fmaf(da[4 * qx], t2[0], fmaf(la[4 * qx], t2[1], hs));
          ss = fmaf(la[4 * qx], t2[2], ss);
        }
        add_fe(i, r, hs, ss);
      }
    }
  } else {
    // ---- F x E block, slot form ------------------------------------------------
    // For column r = (v, alpha), v = (t_x, t_y, t_z), the PU factor is
    // phi_v = 1/8 l_tx(x) l_ty(y) l_tz(z) with l_0 = 1 - xi, l_1 = 1 + xi, so
    //   8 H_ir = <w V Psi, M M M> + sum_d [ 1/2 (2/h_d)^2 s_td <w Psi, D0 on d, M elsewhere>
    //                                     + 1/2 (2/h_d) <w d_d Psi, D on d, M elsewhere> ],
    //   8 S_ir = <w Psi, M M M>,
    // i = (a, b, c), with the 1D factors M = L_a l_t, D = L'_a l_t, D0 = L'_a
    // (derivatives in xi) and s_t = -1, +1 for t = 0, 1.  All eight vertices of
    // a slot share the projections of its four fields (w Psi, w V Psi,
    // w d_d Psi), contracted z, y, x:
    //   z: Z_S, Z_x, Z_y on M_z; Z_V = M_z (w V Psi) + D_z (1/2 (2/h_z) w d_z Psi)
    //      + D0_z (1/2 (2/h_z)^2 s_tz w Psi)                    (8 (c, t_z) each)
    //   y: W1 = M_y Z_V + 1/2 (2/h_y) D_y Z_y + 1/2 (2/h_y)^2 s_ty D0_y Z_S,
    //      W3 = M_y Z_x, WS = M_y Z_S                          (64 (b t_y, c t_z))
    //   x: 8 H = M_x W1 + 1/2 (2/h_x) D_x W3 + 1/2 (2/h_x)^2 s_tx D0_x WS,
    //      8 S = M_x WS                                          (512 per slot)
    // about 48 p^3 + 320 p^2 + 2048 p multiply-adds per slot, against
    // 8 (16 p^3 + 48 p^2 + 128 p) plus eight evaluations of b_r per point for
    // the column-by-column projection.
    const int per_s = 36 * p2 + 192 * p;
    const int G = max(1, min(A, E.wfloats / per_s));
    const float hx2 = 0.5f * E.sx, hy2 = 0.5f * E.sy, hz2 = 0.5f * E.sz;   // 1/2 (2/h_d)
    const float hxx = hx2 * E.sx, hyy = hy2 * E.sy, hzz = hz2 * E.sz;       // 1/2 (2/h_d)^2
    for (int s0 = 0; s0 < A; s0 += G) {
      const int Gc = min(G, A - s0);
      float *T1 = E.work;                   // [Gc][p^2][36]: Z_S, Z_x, Z_y, Z_V x (t_z, c), pad
      float *T2 = E.work + Gc * p2 * 36;    // [Gc][p][b + 4 t_y][24]: W1, W3, WS x (t_z, c)
      __syncthreads();
      // z: one thread per (slot, qx, qy, t_z)
      for (int it = tid; it < Gc * p2 * 2; it += ST_NT) {
        const int tz = it & 1, col = it >> 1;
        const int g = dp2.div(col), qxy = col - g * p2, slot = s0 + g;
        const float f0s = tz ? hzz : -hzz;
        float4 zs = make_float4(0.f, 0.f, 0.f, 0.f), zx = zs, zy = zs, zv = zs;
        for (int qz = 0; qz < p; ++qz) {
          const int lq = qxy + p2 * qz;
          const float w = xval(lq).w;
          const float fS = w * psv(lq, slot, 0), fx = w * psv(lq, slot, 1),
                      fy = w * psv(lq, slot, 2), fz = hz2 * (w * psv(lq, slot, 3));
          const float fV = fS * vval(lq), f0 = f0s * fS;
          const float4 M = MT[(2 * pm + qz) * 2 + tz], D = DT[(2 * pm + qz) * 2 + tz],
                       D0 = D0T[2 * pm + qz];
          zs.x = fmaf(M.x, fS, zs.x);
          zs.y = fmaf(M.y, fS, zs.y);
          zs.z = fmaf(M.z, fS, zs.z);
          zs.w = fmaf(M.w, fS, zs.w);
          zx.x = fmaf(M.x, fx, zx.x);
          zx.y = fmaf(M.y, fx, zx.y);
          zx.z = fmaf(M.z, fx, zx.z);
          zx.w = fmaf(M.w, fx, zx.w);
          zy.x = fmaf(M.x, fy, zy.x);
          zy.y = fmaf(M.y, fy, zy.y);
          zy.z = fmaf(M.z, fy, zy.z);
          zy.w = fmaf(M.w, fy, zy.w);
          zv.x = fmaf(M.x, fV, fmaf(D.x, fz, fmaf(D0.x, f0, zv.x)));
          zv.y = fmaf(M.y, fV, fmaf(D.y, fz, fmaf(D0.y, f0, zv.y)));
          zv.z = fmaf(M.z, fV, fmaf(D.z, fz, fmaf(D0.z, f0, zv.z)));
          zv.w = fmaf(M.w, fV, fmaf(D.w, fz, fmaf(D0.w, f0, zv.w)));
        }
        float4 *t1 = reinterpret_cast<float4 *>(T1 + (size_t)col * 36 + tz * 4);
        t1[0] = zs;
        t1[2] = zx;
        t1[4] = zy;
        t1[6] = zv;
      }
      __syncthreads();
      // y: one thread per (slot, qx, b, t_y, t_z); four c each
      for (int it = tid; it < Gc * p * 16; it += ST_NT) {
        const int tz = it & 1, bty = (it >> 1) & 7, rest = it >> 4;   // rest = g p + qx
        const int g = dp.div(rest), qx = rest - g * p;
        const int b = bty & 3, ty = bty >> 2;
        const float c0s = ty ? hyy : -hyy;
        float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f), w3 = w1, ws = w1;
        const float4 *t1 = reinterpret_cast<const float4 *>(T1 + (size_t)(g * p2 + qx) * 36) + tz;
        for (int qy = 0; qy < p; ++qy, t1 += p * 9) {
          const float4 m4 = MT[(pm + qy) * 2 + ty], d4 = DT[(pm + qy) * 2 + ty], o4 = D0T[pm + qy];
          const float My = b == 0 ? m4.x : (b == 1 ? m4.y : (b == 2 ? m4.z : m4.w));
          const float Dy = hy2 * (b == 0 ? d4.x : (b == 1 ? d4.y : (b == 2 ? d4.z : d4.w)));
          const float Oy = c0s * (b == 0 ? o4.x : (b == 1 ? o4.y : (b == 2 ? o4.z : o4.w)));
          const float4 zs = t1[0], zx = t1[2], zy = t1[4], zv = t1[6];
          w1.x = fmaf(My, zv.x, fmaf(Dy, zy.x, fmaf(Oy, zs.x, w1.x)));
          w1.y = fmaf(My, zv.y, fmaf(Dy, zy.y, fmaf(Oy, zs.y, w1.y)));
          w1.z = fmaf(My, zv.z, fmaf(Dy, zy.z, fmaf(Oy, zs.z, w1.z)));
          w1.w = fmaf(My, zv.w, fmaf(Dy, zy.w, fmaf(Oy, zs.w, w1.w)));
          w3.x = fmaf(My, zx.x, w3.x);
          w3.y = fmaf(My, zx.y, w3.y);
          w3.z = fmaf(My, zx.z, w3.z);
          w3.w = fmaf(My, zx.w, w3.w);
          ws.x = fmaf(My, zs.x, ws.x);
          ws.y = fmaf(My, zs.y, ws.y);
          ws.z = fmaf(My, zs.z, ws.z);
          ws.w = fmaf(My, zs.w, ws.w);
        }
        float4 *t2 = reinterpret_cast<float4 *>(T2 + ((size_t)rest * 8 + bty) * 24) + tz;
        t2[0] = w1;
        t2[2] = w3;
        t2[4] = ws;
      }
      __syncthreads();
      // x: one thread per (slot, vertex, b, c); the four a, then into both
      // triangles of the columns that exist
      for (int it = tid; it < Gc * 128; it += ST_NT) {
        const int bc = it & 15, v = (it >> 4) & 7, g = it >> 7;
        const int r = E.scol[(s0 + g) * 8 + v];
        if (r < 0) continue;
        const int tx = v & 1, ty = (v >> 1) & 1, tz = v >> 2;
        const int b = bc & 3, c = bc >> 2;
        const float o0s = tx ? hxx : -hxx;
        float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, s0v = 0.f, s1v = 0.f, s2v = 0.f, s3v = 0.f;
        const float *t2 = T2 + (size_t)(g * p * 8 + b + 4 * ty) * 24 + tz * 4 + c;
        for (int qx = 0; qx < p; ++qx, t2 += 8 * 24) {
          const float w1 = t2[0], w3 = hx2 * t2[8], ws = t2[16], wo = o0s * ws;
          const float4 M = MT[qx * 2 + tx], D = DT[qx * 2 + tx], D0 = D0T[qx];
          h0 = fmaf(M.x, w1, fmaf(D.x, w3, fmaf(D0.x, wo, h0)));
          h1 = fmaf(M.y, w1, fmaf(D.y, w3, fmaf(D0.y, wo, h1)));
          h2 = fmaf(M.z, w1, fmaf(D.z, w3, fmaf(D0.z, wo, h2)));
          h3 = fmaf(M.w, w1, fmaf(D.w, w3, fmaf(D0.w, wo, h3)));
          s0v = fmaf(M.x, ws, s0v);
          s1v = fmaf(M.y, ws, s1v);
          s2v = fmaf(M.z, ws, s2v);
          s3v = fmaf(M.w, ws, s3v);
        }
        const float hv[4] = {0.125f * h0, 0.125f * h1, 0.125f * h2, 0.125f * h3};
        const float sv[4] = {0.125f * s0v, 0.125f * s1v, 0.125f * s2v, 0.125f * s3v};
  #pragma unroll
        for (int a = 0; a < 4; ++a) add_fe(a + 4 * b + 16 * c, r, hv[a], sv[a]);
      }
    }
  }

  // ---- E x E block of H (S's is computed by its own kernel) -------------------
  if (!E.wantH) return;
  // ---- E x E block, enrichment-pair form -------------------------------------
  if (E.sp) {
    const int per = 24 * p2 + 66 * p;            // work floats of one pair
    const int fit = max(1, E.wfloats / per);     // the caller checked per <= wfloats
    const int nch = (E.npair + fit - 1) / fit;
    const int npc = (E.npair + nch - 1) / nch;   // pairs per chunk, balanced
    const float *Fy = E.F1 + 6 * pm, *Fx = E.F1;
    const FastDiv dp23(p * 23), d23(23), d66(66);
    for (int c0 = 0; c0 < E.npair; c0 += npc) {
      const int nc = min(npc, E.npair - c0);
      float *T1 = E.work;                        // [nc][p^2][24]: z outputs, pad
      float *T2 = E.work + nc * p2 * 24;         // [nc][p][66]: y outputs
      __syncthreads();
      // z: one thread per (pair, qx, qy) column
      for (int it = tid; it < nc * p2; it += ST_NT) {
        const int g = dp2.div(it), qxy = it - g * p2;
        const int pr = E.pairs[c0 + g], al = pr & 0xff, be = pr >> 8;
        float o[24];
#pragma unroll
        for (int u = 0; u < 24; ++u) o[u] = 0.0f;
        for (int qz = 0; qz < p; ++qz) {
          const int lq = qxy + p2 * qz;
          const float4 x4 = xval(lq);
          const float vq = vval(lq);
          const float a0 = psv(lq, al, 0), a1 = psv(lq, al, 1), a2 = psv(lq, al, 2),
                      a3 = psv(lq, al, 3);
          const float b0 = psv(lq, be, 0), b1 = psv(lq, be, 1), b2 = psv(lq, be, 2),
                      b3 = psv(lq, be, 3);
          const float wa = x4.w * a0, wb = x4.w * b0;
          const float fA = wa * b0;
          const float fE = fmaf(vq, fA, 0.5f * x4.w * fmaf(a1, b1, fmaf(a2, b2, a3 * b3)));
          const float l0 = 1.0f - x4.z, l1 = 1.0f + x4.z;
          const float u0 = l0 * l0, u1 = l0 * l1, u2 = l1 * l1;
          const float f3[4] = {wb * a1, wa * b1, wb * a2, wa * b2};   // B_x C_x B_y C_y
          o[0] = fmaf(fA, u0, o[0]);
          o[1] = fmaf(fA, u1, o[1]);
          o[2] = fmaf(fA, u2, o[2]);
          o[3] += fA;
          o[4] = fmaf(fE, u0, o[4]);
          o[5] = fmaf(fE, u1, o[5]);
          o[6] = fmaf(fE, u2, o[6]);
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            o[7 + 3 * f] = fmaf(f3[f], u0, o[7 + 3 * f]);
            o[8 + 3 * f] = fmaf(f3[f], u1, o[8 + 3 * f]);
            o[9 + 3 * f] = fmaf(f3[f], u2, o[9 + 3 * f]);
          }
          const float Bz = wb * a3, Cz = wa * b3;
          o[19] = fmaf(Bz, l0, o[19]);
          o[20] = fmaf(Bz, l1, o[20]);
          o[21] = fmaf(Cz, l0, o[21]);
          o[22] = fmaf(Cz, l1, o[22]);
        }
        float4 *t1 = reinterpret_cast<float4 *>(T1 + (size_t)it * 24);
#pragma unroll
        for (int u = 0; u < 6; ++u) t1[u] = make_float4(o[4 * u], o[4 * u + 1], o[4 * u + 2], o[4 * u + 3]);
      }
      __syncthreads();
      // y: one thread per (pair, qx, z row); 2-4 outputs each
      for (int it = tid; it < nc * p * 23; it += ST_NT) {
        const int g = dp23.div(it), rem = it - g * p * 23;
        const int qx = d23.div(rem), a = rem - qx * 23;
        int j0, f0, n;
        sp_yrow(a, j0, f0, n);
        const float *t1 = T1 + ((size_t)g * p2 + qx) * 24 + a;
        const float *fy0 = Fy + f0 * pm, *fy1 = fy0 + pm, *fy2 = Fy + min(f0 + 2, 5) * pm,
                    *fy3 = Fy + 3 * pm;
        float c0v = 0.0f, c1v = 0.0f, c2v = 0.0f, c3v = 0.0f;
        for (int qy = 0; qy < p; ++qy) {
          const float t = t1[qy * p * 24];
          c0v = fmaf(fy0[qy], t, c0v);
          c1v = fmaf(fy1[qy], t, c1v);
          c2v = fmaf(fy2[qy], t, c2v);
          c3v = fmaf(fy3[qy], t, c3v);
        }
        float *t2 = T2 + (g * p + qx) * 66;
        t2[j0] = c0v;
        t2[j0 + 1] = c1v;
        if (n > 2) t2[j0 + 2] = c2v;
        if (a < 3) t2[9 + a] = c3v;
      }
      __syncthreads();
      // x: one thread per (pair, y row); 2-4 projections each, the (sub)cells
      // of the element add up
      for (int it = tid; it < nc * 66; it += ST_NT) {
        const int g = d66.div(it), j = it - g * 66;
        int i0, f0, n;
        sp_xrow(j, i0, f0, n);
        const float *t2 = T2 + (size_t)g * p * 66 + j;
        const float *fx0 = Fx + f0 * pm, *fx1 = fx0 + pm, *fx2 = Fx + min(f0 + 2, 5) * pm,
                    *fx3 = Fx + 3 * pm;
        float c0v = 0.0f, c1v = 0.0f, c2v = 0.0f, c3v = 0.0f;
        for (int qx = 0; qx < p; ++qx) {
          const float t = t2[qx * 66];
          c0v = fmaf(fx0[qx], t, c0v);
          c1v = fmaf(fx1[qx], t, c1v);
          c2v = fmaf(fx2[qx], t, c2v);
          c3v = fmaf(fx3[qx], t, c3v);
        }
        float *pe = E.PE + (c0 + g) * 189;
        pe[i0] += c0v;
        pe[i0 + 1] += c1v;
        if (n > 2) pe[i0 + 2] += c2v;
        if (j < 9) pe[27 + j] += c3v;
      }
    }
    return;
  }

  // ---- E x E block over this (sub)cell's points --------------------------------
  float h16[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) h16[u] = 0.0f;
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
          }
        }
      }
    }
  }
  // the PG point groups meet in shared memory, one group after the other (a
  // fixed order, so the block is the same on every call)
  for (int g = 0; g < E.PG; ++g) {
    if (E.act && E.pg == g) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) E.HE[(4 * E.rb + i) * ne8 + 4 * E.sb + j] += h16[i * 4 + j];
    }
    __syncthreads();
  }
}

template <bool BLOCH>
__global__ void __maxnreg__(ST_MAXREG) k_strip_sf(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const double *__restrict__ V, const int32_t *__restrict__ partoff,
    const int32_t *__restrict__ part_p, const int32_t *__restrict__ part_q,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ ecol,
    const int32_t *__restrict__ aoff, const int64_t *__restrict__ toff32,
    const float *__restrict__ psi, const int64_t *__restrict__ soff,
    const int32_t *__restrict__ smap, float sx, float sy, float sz, int pm, int wfloats,
    int sfloats, int eefloats, int amax, int what, double *__restrict__ H,
    double *__restrict__ S,
    unsigned *err, const uint8_t *__restrict__ eshift, PhaseTab ph, double *__restrict__ Hi,
    double *__restrict__ Si, const int8_t *__restrict__ eeform,
    const int32_t *__restrict__ citems) {
  extern __shared__ float4 sm_st4[];
  __shared__ float s_phr[8], s_phi[8];
  // work item: element order[k0], its (sub)cells [cb, ce) (all of them
  // without a work list); partial blocks of one element meet in the atomics
  int k0 = blockIdx.x, cb = 0, ce = 1 << 30;
  if (citems) {
    k0 = citems[3 * blockIdx.x];
    cb = citems[3 * blockIdx.x + 1];
    ce = citems[3 * blockIdx.x + 2];
  }
  const int e = order[k0], tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  StripElem E;
  if (BLOCH) {
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        s_phr[c] = (float)ph.re[c];
        s_phi[c] = (float)ph.im[c];
      }
    }
    E.esh = eshift + doff[e];
    E.phr = s_phr;
    E.phi = s_phi;
    E.Hi = Hi;
    E.Si = Si;
  }
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

  // shared memory: [T4: 18 pm float4][stage: sfloats][work: wfloats]
  //                [E x E: eefloats][F1: 18 pm][ecs: 64 ints][pairs: 36 ints]
  //                [scol: 8 amax ints]
  // E x E area: HE ([ne8][ne8], entries r <= s; direct form) or
  // the pair projections [npair][189] (enrichment-pair form)
  float4 *T4 = sm_st4;
  E.T4 = T4;
  E.stage = reinterpret_cast<float *>(T4 + 18 * pm);
  E.work = E.stage + sfloats;
  E.HE = E.work + wfloats;
  E.PE = E.HE;
  float *F1 = E.HE + eefloats;
  E.F1 = F1;
  int *ecs = reinterpret_cast<int *>(F1 + 18 * pm);
  int *pairs = ecs + 64;
  int *scol = pairs + 36;
  E.ecs = ecs;
  E.pairs = pairs;
  E.scol = scol;
  if (E.A > amax) {
    if (tid == 0) atomicOr(err, DEVERR_SHAPE);
    return;
  }
  for (int o = tid; o < E.A * 8; o += ST_NT) scol[o] = -1;
  __syncthreads();
  if (tid < ne) {
    const int c = ecol[(doff[e] - 64ll * e) + tid];
    ecs[tid] = c;
    scol[c] = tid;   // code = slot * 8 + vertex
  }

  // E x E form: the pair form when the element has at most 8 slots, its
  // projections fit the E x E area, every (sub)cell's pair work fits the work
  // area, and -- unless the autotuner chose a form for the element's class
  // (eeform 1: pair form, 2: direct) -- its estimated operation count (per
  // pair and point: ~56 in z, ~200 / p in y, ~570 / p^2 in x) is below the
  // direct one (~100 per 4 x 4 tile and point, plus ~35 per column and point
  // for the chunk tables)
  {
    const int A = E.A, npair = A * (A + 1) / 2;
    bool sp = A <= 8 && npair * 189 <= eefloats;
    for (int k = partoff[e]; k < partoff[e + 1] && sp; ++k) {
      const int p = part_p[k];
      sp = 24 * p * p + 66 * p <= wfloats;
    }
    const int form = eeform ? eeform[e] : 0;
    if (sp && form == 2) sp = false;
    if (sp && form != 1) {
      const int p = part_p[partoff[e]];
      const int nb = ne8 >> 2;
      const long long cost_sp = (long long)npair * (56 * p * p * p + 200 * p * p + 570 * p + 2835);
      const long long cost_dir = (long long)(nb * (nb + 1) / 2 * 100 + 35 * ne8) * p * p * p;
      sp = cost_sp < cost_dir;
    }
    E.sp = sp;
    E.npair = sp ? npair : 0;
    if (sp && tid < A) {
      int k = tid * A - tid * (tid - 1) / 2;   // pairs (alpha, beta), alpha <= beta, alpha-major
      for (int b = tid; b < A; ++b) pairs[k++] = tid | (b << 8);
    }
  }
  // F x E form: the slot form unless its per-slot y and x stages outweigh
  // the column form's per-column evaluations of b_r (first (sub)cell's p)
  {
    const long long p = part_p[partoff[e]], p2 = p * p, p3 = p2 * p;
    E.fxs = (long long)E.A * (48 * p3 + 320 * p2 + 2048 * p) <
            (long long)ne * (41 * p3 + 48 * p2 + 128 * p);
  }
  const int ee_zero = E.sp ? E.npair * 189 : ne8 * ne8;
  for (int o = tid; o < ee_zero; o += ST_NT) E.HE[o] = 0.0f;

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

  const int kend = min(partoff[e + 1], partoff[e] + ce);
  for (int k = partoff[e] + cb; k < kend; ++k) {
    const int p = part_p[k];
    const int p2 = p * p, p3 = p2 * p;
    if (p > pm || 36 * p2 + 192 * p > wfloats || ST_KC * (4 * ne8 + 1) > wfloats) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    E.p = p;
    E.qs = part_q[k];
    const int P = p3 | 1, A = E.A, qs = E.qs;
    const bool staged = ((A * 4 * P + 3) & ~3) + 5 * p3 <= sfloats;
    __syncthreads();   // previous users of stage/work/T4 are done
    if (staged) {   // Psi transposed to [slot][comp][point], pitch P (odd)
      float *stage = E.stage;
      float4 *xd = reinterpret_cast<float4 *>(stage + ((A * 4 * P + 3) & ~3));
      float *vd = reinterpret_cast<float *>(xd + p3);
      const int blk0 = qs >> 3, nblk = ((qs + p3 + 7) >> 3) - blk0;
      const float4 *src = reinterpret_cast<const float4 *>(E.pe + (int64_t)blk0 * A * 32);
      const FastDiv dA8(A * 8);
      // one float4 = 4 points of a row; four loads in flight per thread
      const int nsrc = nblk * A * 8;
      for (int o0 = tid; o0 < nsrc; o0 += 4 * ST_NT) {
        float4 v4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          v4[u] = o0 + u * ST_NT < nsrc ? src[o0 + u * ST_NT] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int o = o0 + u * ST_NT;
          if (o >= nsrc) break;
          const int blk = dA8.div(o), rem = o - blk * (A * 8);
          const int row = rem >> 1;   // slot * 4 + comp
          const int qb = (blk0 + blk) * 8 + (rem & 1) * 4 - qs;
          float *d = stage + row * P;
          if (qb >= 0 && qb < p3) d[qb] = v4[u].x;
          if (qb + 1 >= 0 && qb + 1 < p3) d[qb + 1] = v4[u].y;
          if (qb + 2 >= 0 && qb + 2 < p3) d[qb + 2] = v4[u].z;
          if (qb + 3 >= 0 && qb + 3 < p3) d[qb + 3] = v4[u].w;
        }
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
      const float xd = d == 0 ? x4.x : (d == 1 ? x4.y : x4.z);
      float L[4], dL[4];
      lag3vd(xd, L, dL);
      const float l0 = 1.0f - xd, l1 = 1.0f + xd;
      T4[(d * pm + t) * 2] = make_float4(L[0] * l0, L[1] * l0, L[2] * l0, L[3] * l0);
      T4[(d * pm + t) * 2 + 1] = make_float4(L[0] * l1, L[1] * l1, L[2] * l1, L[3] * l1);
      T4[6 * pm + (d * pm + t) * 2] = make_float4(dL[0] * l0, dL[1] * l0, dL[2] * l0, dL[3] * l0);
      T4[6 * pm + (d * pm + t) * 2 + 1] =
          make_float4(dL[0] * l1, dL[1] * l1, dL[2] * l1, dL[3] * l1);
      T4[12 * pm + d * pm + t] = make_float4(dL[0], dL[1], dL[2], dL[3]);
      T4[15 * pm + d * pm + t] = make_float4(L[0], L[1], L[2], L[3]);
      float *f1 = F1 + d * 6 * pm + t;
      f1[0] = l0 * l0;
      f1[pm] = l0 * l1;
      f1[2 * pm] = l1 * l1;
      f1[3 * pm] = 1.0f;
      f1[4 * pm] = l0;
      f1[5 * pm] = l1;
    }
    if (staged)
      strip_part<true, BLOCH>(E, H, S);
    else
      strip_part<false, BLOCH>(E, H, S);
  }
  __syncthreads();
  // ---- E x E block of H into the FP64 CSR values, both triangles ----------------
  if (!E.wantH) return;
  const FastDiv dne(ne);
  if (E.sp) {   // entries from the pair projections (slot of r <= slot of s by symmetry)
    const float hx = 0.5f * sx, hy = 0.5f * sy, hz = 0.5f * sz;
    const int A = E.A;
    for (int o = tid; o < ne * ne; o += ST_NT) {
      const int r = dne.div(o), sc = o - r * ne;
      int cr = ecs[r], cs = ecs[sc];
      if ((cr >> 3) > (cs >> 3)) {
        const int t = cr;
        cr = cs;
        cs = t;
      }
      const int al = cr >> 3, be = cs >> 3;
      const float *P = E.PE + (al * A - al * (al - 1) / 2 + (be - al)) * 189;
      const int bx = cr & 1, by = (cr >> 1) & 1, bz = (cr >> 2) & 1;
      const int cx = cs & 1, cy = (cs >> 1) & 1, cz = (cs >> 2) & 1;
      const float px = bx ? 1.0f : -1.0f, py = by ? 1.0f : -1.0f, pz = bz ? 1.0f : -1.0f;
      const float qx = cx ? 1.0f : -1.0f, qy = cy ? 1.0f : -1.0f, qz = cz ? 1.0f : -1.0f;
      const int kx = bx + cx, ky = by + cy, kz = bz + cz;
      const int kzy = kz * 3 + ky;
      float h = P[54 + kzy * 3 + kx];
      h = fmaf(hx * sx * px * qx, P[27 + kzy], h);
      h = fmaf(hy * sy * py * qy, P[36 + kz * 3 + kx], h);
      h = fmaf(hz * sz * pz * qz, P[45 + ky * 3 + kx], h);
      h = fmaf(hx * px, P[99 + kzy * 2 + cx], h);
      h = fmaf(hx * qx, P[81 + kzy * 2 + bx], h);
      h = fmaf(hy * py, P[135 + (kz * 2 + cy) * 3 + kx], h);
      h = fmaf(hy * qy, P[117 + (kz * 2 + by) * 3 + kx], h);
      h = fmaf(hz * pz, P[171 + (cz * 3 + ky) * 3 + kx], h);
      h = fmaf(hz * qz, P[153 + (bz * 3 + ky) * 3 + kx], h);
      const int slot = E.m[(64 + r) * E.n + 64 + sc];
      const float hv = h * (1.0f / 64.0f);
      if (BLOCH) {
        float pr, pi;
        pair_phase(E, E.esh[64 + r], E.esh[64 + sc], pr, pi);
        atomicAdd(H + slot, (double)(hv * pr));
        atomicAdd(E.Hi + slot, (double)(hv * pi));
      } else {
        atomicAdd(H + slot, (double)hv);
      }
    }
    return;
  }
  for (int o = tid; o < ne * ne; o += ST_NT) {
    const int r = dne.div(o), sc = o - r * ne;
    const int lo = min(r, sc), hi = max(r, sc);
    const int slot = E.m[(64 + r) * E.n + 64 + sc];
    if (BLOCH) {
      float pr, pi;
      pair_phase(E, E.esh[64 + r], E.esh[64 + sc], pr, pi);
      const float hv = E.HE[lo * ne8 + hi];
      atomicAdd(H + slot, (double)(hv * pr));
      atomicAdd(E.Hi + slot, (double)(hv * pi));
    } else {
      atomicAdd(H + slot, (double)E.HE[lo * ne8 + hi]);
    }
  }
}

}  // namespace

// Shared-memory floats of the strip kernel's work area: the F x E
// intermediates of one enrichment slot (36 p^2 + 192 p) for every per-axis
// count in `pmask`, or one E x E chunk table for enrichment count (rounded to
// 8) ne8; slots are grouped as far as the area allows.
static int strip_work_floats(uint32_t pmask, int ne8) {
  int w = ST_KC * (4 * ne8 + 1);
  for (int p = 1; p < 32; ++p) {
    if (!(pmask & (1u << p))) continue;
    w = std::max(w, 36 * p * p + 192 * p);
  }
  return (w + 3) & ~3;
}

// ph == nullptr: Gamma point; else the Bloch scatter into (H, Hi), (S, Si)
// The strip kernel over `count` elements listed on the device at `ord`
// (host copy `hord` for the launch sizes).
// With `citems` (the context's (sub)cell-range list of all strip elements,
// `nitems` items) the grid runs over the list instead.
static pufe_status strip_launch_list(pufe_ctx *ctx, const double *V, int what, double *H,
                                     double *S, const int32_t *ord, const int32_t *hord, int count,
                                     cudaStream_t st, const PhaseTab *ph, double *Hi, double *Si,
                                     const int32_t *citems = nullptr, int nitems = 0) {
  if (count <= 0) return PUFE_OK;
  const unsigned grid = citems ? (unsigned)nitems : (unsigned)count;
  if (grid == 0) return PUFE_OK;
  auto &D = ctx->d;
  int ne8 = 8;
  for (int k = 0; k < count; ++k) ne8 = std::max(ne8, (ctx->n_e[hord[k]] - 64 + 7) & ~7);
  const int sneed = ctx->strip_stage;
  if (ne8 > 64) return fail(PUFE_EINVAL, "strip kernel takes n_e <= 128");
  const int pm = std::max(1, ctx->max_part_p);
  {   // FastDiv preconditions, x d < 2^32 for the largest index of each division
    const int64_t p2 = (int64_t)pm * pm, p3 = p2 * pm, A = ne8;
    const int64_t xd[][2] = {
        {64 * p2, p2},                                      // slot-form z stage
        {64 * pm, pm},                                      // slot-form y stage
        {36 * 23 * pm, 23 * pm},                            // pair-form y stage
        {(int64_t)ST_KC * ne8, ne8},                        // E x E chunk table
        {((p3 + 7) / 8 + 1) * 8 * A, 8 * A},                // Psi staging
        {(int64_t)ne8 * ne8, ne8}};                         // E x E scatter
    for (auto &v : xd)
      if (v[0] * v[1] >= (int64_t(1) << 32))
        return fail(PUFE_EINVAL, "strip kernel: index range beyond its 32-bit divisions");
  }
  const int wf = strip_work_floats(ctx->strip_pmask, ne8);
  const int sf = (sneed + 3) & ~3;
  const int ee = std::max(ne8 * ne8, 189 * ctx->strip_npair_max);
  int amax = 1;
  for (int k = 0; k < count; ++k) amax = std::max(amax, (int)ctx->n_slot[hord[k]]);
  const size_t sm =
      ((size_t)72 * pm + sf + wf + ee + 18 * pm + 64 + 36 + 8 * amax) * sizeof(float);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "strip kernel: shared memory above 227 KB");
  const float sx = (float)(2.0 / ctx->h[0]), sy = (float)(2.0 / ctx->h[1]),
              sz = (float)(2.0 / ctx->h[2]);
  if (ph) {
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_strip_sf<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_strip_sf<true><<<grid, ST_NT, sm, st>>>(
        ord, D.qoff, D.qpoff, D.qdat, V, D.partoff, D.part_p, D.part_q, D.doff,
        D.ecol, D.aoff, D.toff32, D.psi32, D.soff, D.smap, sx, sy, sz, pm, wf, sf, ee, amax, what, H, S,
        D.err, D.eshift, *ph, Hi, Si, D.eeform, citems);
  } else {
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_strip_sf<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_strip_sf<false><<<grid, ST_NT, sm, st>>>(
        ord, D.qoff, D.qpoff, D.qdat, V, D.partoff, D.part_p, D.part_q, D.doff,
        D.ecol, D.aoff, D.toff32, D.psi32, D.soff, D.smap, sx, sy, sz, pm, wf, sf, ee, amax, what, H, S,
        D.err, nullptr, PhaseTab{}, nullptr, nullptr, D.eeform, citems);
  }
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

static pufe_status strip_launch(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                                int first, int count, cudaStream_t st, const PhaseTab *ph,
                                double *Hi, double *Si) {
  // all strip elements: over the (sub)cell-range work list, whose items
  // index `order` from its start
  const bool all = first == ctx->n_big && first + count == ctx->nelem && ctx->d.citems;
  return strip_launch_list(ctx, V, what, H, S, ctx->d.order + (all ? 0 : first),
                           ctx->order.data() + first, count, st, ph, Hi, Si,
                           all ? ctx->d.citems : nullptr, all ? ctx->n_citems : 0);
}

// ---------------------------------------------------------------------------
// Autotuner of the E x E form.  Strip elements (64 < n_e <= 128) are grouped
// into classes by (n_e, slots, points per axis of every (sub)cell); for each
// class where both forms apply, the strip kernel is timed on the class's
// elements (up to 256 of them) with the enrichment-pair form and with the
// direct 4 x 4 tiles forced, and the faster is kept for every element of the
// class.  With PUFE_AUTOTUNE_CACHE naming a file, decisions found there (one
// line per class: key, form) are taken without timing, and new ones are
// appended.
// ---------------------------------------------------------------------------
pufe_status autotune_strip(pufe_ctx *ctx, int *ntuned, cudaStream_t st) {
  auto &D = ctx->d;
  if (ntuned) *ntuned = 0;
  if (!ctx->tabulated32) return fail(PUFE_ESTATE, "call pufe_tabulate(PUFE_TF32X3) first");
  // classes
  std::map<std::string, std::vector<int32_t>> cls;
  std::vector<int32_t> pbeg(ctx->nelem + 1, 0);
  for (int64_t e = 0; e < ctx->nelem; ++e) {
    const int n = ctx->n_e[e];
    if (n <= 64 || n > 128) continue;
    const int A = ctx->n_slot[e];
    if (A > 8) continue;   // the pair form takes at most 8 slots
    std::string key = "ne=" + std::to_string(n) + ",A=" + std::to_string(A) + ",p=";
    for (size_t k = 0; k < ctx->part_p_host[e].size(); ++k)
      key += (k ? "." : "") + std::to_string(ctx->part_p_host[e][k]);
    cls[key].push_back((int32_t)e);
  }
  std::map<std::string, int> cache;
  const char *path = std::getenv("PUFE_AUTOTUNE_CACHE");
  if (path && *path) {
    std::ifstream in(path);
    std::string k;
    int f;
    while (in >> k >> f)
      if (f == 1 || f == 2) cache[k] = f;
  }
  double *H = nullptr, *S = nullptr, *V = nullptr;
  int32_t *dord = nullptr;
  cudaEvent_t ea = nullptr, eb = nullptr;
  auto cleanup = [&]() {
    if (H) cudaFree(H);
    if (S) cudaFree(S);
    if (V) cudaFree(V);
    if (dord) cudaFree(dord);
    if (ea) cudaEventDestroy(ea);
    if (eb) cudaEventDestroy(eb);
  };
  pufe_status rc = PUFE_OK;
  std::vector<std::pair<std::string, int>> fresh;
  do {
    size_t maxcls = 0;
    for (auto &kv : cls) maxcls = std::max(maxcls, std::min<size_t>(kv.second.size(), 256));
    if (cudaMalloc((void **)&H, std::max<int64_t>(1, ctx->nnz) * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&S, std::max<int64_t>(1, ctx->nnz) * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&V, std::max<int64_t>(1, ctx->nq) * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&dord, std::max<size_t>(1, maxcls) * sizeof(int32_t)) != cudaSuccess ||
        cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(PUFE_ENOMEM, "autotune: scratch allocation failed");
      break;
    }
    if (cudaMemsetAsync(V, 0, ctx->nq * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(H, 0, ctx->nnz * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(S, 0, ctx->nnz * sizeof(double), st) != cudaSuccess) {
      rc = fail(PUFE_ECUDA, "autotune: memset failed");
      break;
    }
    for (auto &kv : cls) {
      int choice = 0;
      auto hit = cache.find(kv.first);
      if (hit != cache.end()) {
        choice = hit->second;
      } else {
        // up to 256 elements spread over the class
        std::vector<int32_t> sel;
        const size_t m = kv.second.size(), take = std::min<size_t>(m, 256);
        for (size_t i = 0; i < take; ++i) sel.push_back(kv.second[i * m / take]);
        if (cudaMemcpy(dord, sel.data(), sel.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
          rc = fail(PUFE_ECUDA, "autotune: copy failed");
          break;
        }
        float best = 0.0f;
        for (int form = 1; form <= 2 && rc == PUFE_OK; ++form) {
          for (int32_t e : sel) ctx->eeform_host[e] = (int8_t)form;
          if (cudaMemcpy(D.eeform, ctx->eeform_host.data(), ctx->nelem, cudaMemcpyHostToDevice) !=
              cudaSuccess) {
            rc = fail(PUFE_ECUDA, "autotune: copy failed");
            break;
          }
          float tmin = 1e30f;
          for (int rep = 0; rep < 4 && rc == PUFE_OK; ++rep) {
            cudaEventRecord(ea, st);
            rc = strip_launch_list(ctx, V, PUFE_WANT_H | PUFE_WANT_S, H, S, dord, sel.data(),
                                   (int)sel.size(), st, nullptr, nullptr, nullptr);
            cudaEventRecord(eb, st);
            if (rc == PUFE_OK && cudaEventSynchronize(eb) == cudaSuccess) {
              float t = 0.0f;
              cudaEventElapsedTime(&t, ea, eb);
              if (rep > 0) tmin = std::min(tmin, t);   // the first launch warms up
            }
          }
          if (form == 1 || tmin < best) {
            best = tmin;
            choice = form;
          }
        }
        if (rc != PUFE_OK) break;
        fresh.push_back({kv.first, choice});
      }
      for (int32_t e : kv.second) ctx->eeform_host[e] = (int8_t)choice;
      if (ntuned) ++*ntuned;
    }
    if (rc != PUFE_OK) break;
    if (cudaMemcpy(D.eeform, ctx->eeform_host.data(), ctx->nelem, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      rc = fail(PUFE_ECUDA, "autotune: copy failed");
      break;
    }
    unsigned flag = 0;
    cudaMemcpy(&flag, D.err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (flag) rc = fail(PUFE_EDEVICE, "autotune: a strip launch reported a device error");
    if (path && *path && !fresh.empty()) {
      std::ofstream out(path, std::ios::app);
      for (auto &kv : fresh) out << kv.first << " " << kv.second << "\n";
    }
  } while (false);
  cleanup();
  return rc;
}

pufe_status launch_strip_sf(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                            int first, int count, cudaStream_t st) {
  return strip_launch(ctx, V, what, H, S, first, count, st, nullptr, nullptr, nullptr);
}

// Mixed-precision H(k), S(k) (Sec. 4, eqs. bloch, strong): the element blocks
// are those of the Gamma-point mixed path; the FE-FE blocks (kinetic and
// overlap constants plus the FP32 V block) are scattered with FP64 phases, the
// enrichment strip's FP32 blocks with FP32 phases, all into FP64 values.
pufe_status launch_assemble_mixed_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *V,
                                        int what, double *H, double *Hi, double *S, double *Si,
                                        cudaStream_t st) {
  if (!ctx->fe_exact)
    return fail(PUFE_EINVAL, "PUFE_TF32X3 needs every (sub)cell rule to have >= 4 points per axis");
  if (ctx->n_big > 0) return fail(PUFE_EINVAL, "the mixed Bloch assembly takes n_e <= 128");
  const size_t bytes = (size_t)ctx->nnz * sizeof(double);
  if (what & PUFE_WANT_H) {
    PUFE_CUDA_TRY(cudaMemsetAsync(H, 0, bytes, st));
    PUFE_CUDA_TRY(cudaMemsetAsync(Hi, 0, bytes, st));
  }
  if (what & PUFE_WANT_S) {
    PUFE_CUDA_TRY(cudaMemsetAsync(S, 0, bytes, st));
    PUFE_CUDA_TRY(cudaMemsetAsync(Si, 0, bytes, st));
  }
  pufe_status e0 = launch_fefe_bloch(ctx, ph, V, what, H, Hi, S, Si, st);
  if (e0 != PUFE_OK) return e0;
  if (what & PUFE_WANT_S) {   // E x E block of S(k) in FP64 with FP64 phases
    pufe_status e1 = launch_see(ctx, &ph, S, Si, st);
    if (e1 != PUFE_OK) return e1;
  }
  return strip_launch(ctx, (what & PUFE_WANT_H) ? V : nullptr, what, H, S, 0, (int)ctx->nelem, st,
                      &ph, Hi, Si);
}

// ---------------------------------------------------------------------------
// Enrichment strip of the adjoint of V -> H (mixed path, n_e <= 128).
//
// dL/dV_q = w_q b_q^T Hbar_e b_q; the FE-FE form is done by k_adjoint_fefe
// (which stores Vbar), this kernel adds the enrichment terms
//   w_q [ sum_{r in E} sum_{j in F} (Hbar_rj + Hbar_jr) b_r phi_j
//         + sum_{r, s in E} Hbar_rs b_r b_s ].
// With b_r = phi_v Psi_alpha and trilinear phi_v = 1/8 prod_d (1 + s_d x_d),
// both sums regroup by enrichment slot, so every point needs only Psi values:
//   F x E:  sum_alpha Psi_alpha(q) G_alpha(q),
//           G_alpha = sum K_alpha[c tz][b ty][a tx] m_{c,tz}(z) m_{b,ty}(y) m_{a,tx}(x),
//           m_{a,t}(x) = L_a(x) (1 -+ x),
//           K_alpha = (Hbar_rj + Hbar_jr) / 8 for r = (v(tx,ty,tz), alpha), j = a + 4b + 16c;
//   E x E:  sum_{alpha <= beta} Psi_alpha Psi_beta P_ab(q),
//           P_ab = sum_k D_ab[kz ky kx] u_kz(z) u_ky(y) u_kx(x),  u_k as in the assembly,
//           D_ab[k] = 1/64 sum over vertex pairs (v, v') with b_d + b'_d = k_d of
//                     Hbar_rs (+ Hbar_sr when alpha != beta).
// G and P are evaluated on each p^3 (sub)cell axis by axis (x, then y, then
// z at the point): 8 and 3 multiply-adds per point and slot or pair, against
// 84 per column and point for the direct FE sum.  FP32 with round to nearest.
// ---------------------------------------------------------------------------
namespace {

constexpr int AJ_NT = 256;
constexpr int AJ_W = 4096;   // work floats: x and y stage outputs of one chunk, or the E x E block

template <bool BLOCH>
__global__ void __launch_bounds__(AJ_NT, 4) k_adjoint_strip_sf(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const double *__restrict__ w, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const int32_t *__restrict__ partoff, const int32_t *__restrict__ part_p,
    const int32_t *__restrict__ part_q, const int64_t *__restrict__ soff,
    const int32_t *__restrict__ smap, const double *__restrict__ Hbar, int pm, int cfloats,
    double *__restrict__ Vbar, unsigned *err, BlochCot bc) {
  extern __shared__ float4 sm_aj4[];
  const int e = order[blockIdx.x], tid = threadIdx.x;
  const int n = (int)(doff[e + 1] - doff[e]);
  const int ne = n - 64;
  if (ne <= 0) return;   // FE-only element: Vbar is already complete
  const int A = aoff[e + 1] - aoff[e], npair = A * (A + 1) / 2;
  int p3max = 0, pmax = 0;
  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    pmax = max(pmax, part_p[k]);
    p3max = max(p3max, part_p[k] * part_p[k] * part_p[k]);
  }
  if (!adjoint_sf_fits(A, pmax)) return;   // left to the direct kernel
  if (n > 128 || pmax > pm || A * 512 + npair * 27 + A * p3max > cfloats) {
    if (tid == 0) atomicOr(err, DEVERR_SHAPE);
    return;
  }
  // shared memory: [K: A*512][D: npair*27][Ps: A*p3max][cfloats end]
  //                [M1: 3*8*pm][U1: 3*3*pm][work: AJ_W][cmap: A*8 ints][pairs: npair ints]
  float *K = reinterpret_cast<float *>(sm_aj4);
  float *Dp = K + A * 512;
  float *Ps = Dp + npair * 27;
  float *M1 = K + cfloats;
  float *U1 = M1 + 24 * pm;
  float *work = U1 + 9 * pm;
  int *cmap = reinterpret_cast<int *>(work + AJ_W);
  int *pairs = cmap + A * 8;
  const int64_t q0 = qoff[e];
  const int32_t *m = smap + soff[e];
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  const int32_t *ec = ecol + (doff[e] - 64ll * e);

  // column of (slot, vertex), -1 where the element has none; pair list
  for (int o = tid; o < A * 8; o += AJ_NT) cmap[o] = -1;
  if (tid < A) {
    int k = tid * A - tid * (tid - 1) / 2;
    for (int b = tid; b < A; ++b) pairs[k++] = tid | (b << 8);
  }
  __syncthreads();
  if (tid < ne) cmap[ec[tid]] = tid;   // code = slot * 8 + vertex
  __syncthreads();
  // coefficients from Hbar.  The CSR values are gathered with eight
  // independent (map, value) load chains in flight per thread, each half of
  // K with the lanes of a warp along one CSR row: Hbar_rj (row of enrichment
  // r, FE columns j) first, then Hbar_jr (row of FE j, enrichment columns r)
  // added in; the E x E block goes into the work area
  for (int o = tid; o < A * 512; o += AJ_NT) K[o] = 0.0f;   // absent vertices stay 0
  __syncthreads();
  for (int half = 0; half < 2; ++half) {
    for (int o0 = tid; o0 < ne * 64; o0 += 8 * AJ_NT) {
      int s1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int o = o0 + u * AJ_NT;
        const int r = half ? o % ne : o >> 6, j = half ? o / ne : o & 63;
        s1[u] = o < ne * 64 ? m[half ? j * n + 64 + r : (64 + r) * n + j] : 0;
      }
      double h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) h[u] = o0 + u * AJ_NT < ne * 64 ? Hbar[s1[u]] : 0.0;
      if (BLOCH) {   // at a wavevector: the phased real part
        double hi[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) hi[u] = o0 + u * AJ_NT < ne * 64 ? bc.Hi[s1[u]] : 0.0;
        const uint8_t *esh = bc.eshift + doff[e];
        for (int u = 0; u < 8; ++u) {
          const int o = o0 + u * AJ_NT;
          if (o >= ne * 64) break;
          const int r = half ? o % ne : o >> 6, j = half ? o / ne : o & 63;
          h[u] = half ? cot_entry(h[u], hi[u], esh[j], esh[64 + r], bc.ph)
                      : cot_entry(h[u], hi[u], esh[64 + r], esh[j], bc.ph);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int o = o0 + u * AJ_NT;
        if (o >= ne * 64) break;
        const int r = half ? o % ne : o >> 6, j = half ? o / ne : o & 63;
        const int code = ec[r], v = code & 7;
        const int atx = 2 * (j & 3) + (v & 1), bty = 2 * ((j >> 2) & 3) + ((v >> 1) & 1),
                  ctz = 2 * (j >> 4) + (v >> 2);
        float *kk = K + (code >> 3) * 512 + ctz * 64 + bty * 8 + atx;
        *kk = half ? *kk + (float)(0.125 * h[u]) : (float)(0.125 * h[u]);
      }
    }
    __syncthreads();
  }
  float *HE = work;   // [ne][ne]: Hbar_rs, r, s in E
  for (int o0 = tid; o0 < ne * ne; o0 += 8 * AJ_NT) {
    int s1[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int o = o0 + u * AJ_NT, r = o / ne, sc = o - r * ne;
      s1[u] = o < ne * ne ? m[(64 + r) * n + 64 + sc] : 0;
    }
    double h[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) h[u] = o0 + u * AJ_NT < ne * ne ? Hbar[s1[u]] : 0.0;
    if (BLOCH) {
      double hi[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) hi[u] = o0 + u * AJ_NT < ne * ne ? bc.Hi[s1[u]] : 0.0;
      const uint8_t *esh = bc.eshift + doff[e] + 64;
      for (int u = 0; u < 8; ++u) {
        const int o = o0 + u * AJ_NT, r = o / ne, sc = o - r * ne;
        if (o < ne * ne) h[u] = cot_entry(h[u], hi[u], esh[r], esh[sc], bc.ph);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (o0 + u * AJ_NT < ne * ne) HE[o0 + u * AJ_NT] = (float)h[u];
  }
  __syncthreads();
  for (int o = tid; o < npair * 27; o += AJ_NT) {
    const int pi = o / 27, k = o - pi * 27;
    const int al = pairs[pi] & 0xff, be = pairs[pi] >> 8;
    const int kd[3] = {k % 3, (k / 3) % 3, k / 9};   // x, y, z
    float sum = 0.0f;
    for (int v = 0; v < 8; ++v) {
      int v2 = 0;
      bool ok = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int b2 = kd[d] - ((v >> d) & 1);
        ok = ok && (b2 == 0 || b2 == 1);
        v2 |= (b2 & 1) << d;
      }
      if (!ok) continue;
      const int r = cmap[al * 8 + v], sc = cmap[be * 8 + v2];
      if (r < 0 || sc < 0) continue;
      sum += HE[r * ne + sc];
      if (al != be) sum += HE[sc * ne + r];
    }
    Dp[o] = sum * (1.0f / 64.0f);
  }

  const int nsc_w = AJ_W;
  for (int kp = partoff[e]; kp < partoff[e + 1]; ++kp) {
    const int p = part_p[kp], p2 = p * p, p3 = p2 * p, qs = part_q[kp];
    const FastDiv dp(p), dp2(p2);
    __syncthreads();   // coefficients ready; previous part's readers done
    // Psi values of the (sub)cell's points and the 1D factors per axis
    for (int o0 = tid; o0 < A * p3; o0 += 4 * AJ_NT) {   // four loads in flight per thread
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = o0 + u * AJ_NT, al = o / p3, ql = qs + o - al * p3;
        v[u] = o < A * p3 ? pe[((int64_t)(ql >> 3) * A + al) * 32 + (ql & 7)] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (o0 + u * AJ_NT < A * p3) Ps[o0 + u * AJ_NT] = v[u];
    }
    for (int o = tid; o < 3 * p; o += AJ_NT) {
      const int d = o / p, t = o - d * p;
      const int stride = d == 0 ? 1 : (d == 1 ? p : p2);
      const float4 x4 = qe[qs + t * stride];
      const float xd = d == 0 ? x4.x : (d == 1 ? x4.y : x4.z);
      const float a = xd + 1.0f, b = xd + (1.0f / 3.0f), c = xd - (1.0f / 3.0f), dd = xd - 1.0f;
      const float L[4] = {-0.5625f * b * c * dd, 1.6875f * a * c * dd, -1.6875f * a * b * dd,
                          0.5625f * a * b * c};
      const float l0 = 1.0f - xd, l1 = 1.0f + xd;
#pragma unroll
      for (int aa = 0; aa < 4; ++aa) {
        M1[(d * 8 + 2 * aa) * pm + t] = L[aa] * l0;
        M1[(d * 8 + 2 * aa + 1) * pm + t] = L[aa] * l1;
      }
      U1[(d * 3 + 0) * pm + t] = l0 * l0;
      U1[(d * 3 + 1) * pm + t] = l0 * l1;
      U1[(d * 3 + 2) * pm + t] = l1 * l1;
    }
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // points tid + 256 k (p^3 <= 1024)

    // ---- F x E: slots in chunks ------------------------------------------------
    const int per_s = 64 * p + 8 * p2;
    const int nsc = max(1, nsc_w / per_s);
    for (int s0 = 0; s0 < A; s0 += nsc) {
      const int nc = min(nsc, A - s0);
      float *X = work;                 // [nc][64][p]: (c tz, b ty) rows at x points
      float *Y = work + nc * 64 * p;   // [nc][8][p^2]: c tz rows at (x, y) points
      __syncthreads();
      for (int it = tid; it < nc * 64 * p; it += AJ_NT) {
        const int row = dp.div(it), qx = it - row * p;   // row = g * 64 + (c tz) * 8 + (b ty)
        const float *k8 = K + (s0 * 64 + row) * 8;
        float sum = 0.0f;
#pragma unroll
        for (int t = 0; t < 8; ++t) sum = fmaf(k8[t], M1[t * pm + qx], sum);
        X[it] = sum;
      }
      __syncthreads();
      for (int it = tid; it < nc * 8 * p2; it += AJ_NT) {
        const int row = dp2.div(it), qxy = it - row * p2;   // row = g * 8 + (c tz)
        const int qy = dp.div(qxy), qx = qxy - qy * p;
        const float *x8 = X + row * 8 * p + qx;
        float sum = 0.0f;
#pragma unroll
        for (int t = 0; t < 8; ++t) sum = fmaf(x8[t * p], M1[(8 + t) * pm + qy], sum);
        Y[it] = sum;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int lq = tid + AJ_NT * k;
        if (lq >= p3) break;
        const int qz = lq / p2, qxy = lq - qz * p2;
        float a = acc[k];
        for (int g = 0; g < nc; ++g) {
          const float *y8 = Y + g * 8 * p2 + qxy;
          float gs = 0.0f;
#pragma unroll
          for (int t = 0; t < 8; ++t) gs = fmaf(y8[t * p2], M1[(16 + t) * pm + qz], gs);
          a = fmaf(Ps[(s0 + g) * p3 + lq], gs, a);
        }
        acc[k] = a;
      }
    }

    // ---- E x E: slot pairs in chunks ----------------------------------------------
    const int per_p = 9 * p + 3 * p2;
    const int npc = max(1, nsc_w / per_p);
    for (int c0 = 0; c0 < npair; c0 += npc) {
      const int nc = min(npc, npair - c0);
      float *X = work;                // [nc][9][p]: (kz ky) rows at x points
      float *Y = work + nc * 9 * p;   // [nc][3][p^2]: kz rows at (x, y) points
      __syncthreads();
      for (int it = tid; it < nc * 9 * p; it += AJ_NT) {
        const int row = dp.div(it), qx = it - row * p;   // row = g * 9 + kz * 3 + ky
        const float *d3 = Dp + (c0 * 9 + row) * 3;
        X[it] = fmaf(d3[0], U1[qx], fmaf(d3[1], U1[pm + qx], d3[2] * U1[2 * pm + qx]));
      }
      __syncthreads();
      for (int it = tid; it < nc * 3 * p2; it += AJ_NT) {
        const int row = dp2.div(it), qxy = it - row * p2;   // row = g * 3 + kz
        const int qy = dp.div(qxy), qx = qxy - qy * p;
        const float *x3 = X + row * 3 * p + qx;
        Y[it] = fmaf(x3[0], U1[3 * pm + qy], fmaf(x3[p], U1[4 * pm + qy], x3[2 * p] * U1[5 * pm + qy]));
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int lq = tid + AJ_NT * k;
        if (lq >= p3) break;
        const int qz = lq / p2, qxy = lq - qz * p2;
        const float uz0 = U1[6 * pm + qz], uz1 = U1[7 * pm + qz], uz2 = U1[8 * pm + qz];
        float a = acc[k];
        for (int g = 0; g < nc; ++g) {
          const float *y3 = Y + g * 3 * p2 + qxy;
          const float ps = fmaf(y3[0], uz0, fmaf(y3[p2], uz1, y3[2 * p2] * uz2));
          const int pr = pairs[c0 + g];
          a = fmaf(Ps[(pr & 0xff) * p3 + lq] * Ps[(pr >> 8) * p3 + lq], ps, a);
        }
        acc[k] = a;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int lq = tid + AJ_NT * k;
      if (lq >= p3) break;
      const int64_t q = q0 + qs + lq;
      Vbar[q] += w[q] * (double)acc[k];
    }
  }
}

}  // namespace

pufe_status launch_adjoint_strip_sf(pufe_ctx *ctx, const double *Hbar, double *Vbar, int first,
                                    int count, cudaStream_t st, const BlochCot &bc) {
  if (count <= 0 || ctx->adj_sf_floats == 0) return PUFE_OK;
  auto &D = ctx->d;
  const int pm = std::max(1, ctx->max_part_p);
  // FastDiv preconditions: the divided indices stay below the work area
  // (AJ_W floats), the divisors are p and p^2
  if ((int64_t)AJ_W * pm * pm >= (int64_t(1) << 32))
    return fail(PUFE_EINVAL, "adjoint strip: index range beyond its 32-bit divisions");
  const int cf = (ctx->adj_sf_floats + 3) & ~3;
  const size_t sm = ((size_t)cf + 33 * pm + AJ_W + 16 * 8 + 136) * sizeof(float);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "adjoint strip: shared memory above 227 KB");
  auto kern = bc.Hi ? k_adjoint_strip_sf<true> : k_adjoint_strip_sf<false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<(unsigned)count, AJ_NT, sm, st>>>(
      D.order + first, D.qoff, D.qpoff, D.qdat, D.w, D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
      D.partoff, D.part_p, D.part_q, D.soff, D.smap, Hbar, pm, cf, Vbar, D.err, bc);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

}  // namespace pufe
