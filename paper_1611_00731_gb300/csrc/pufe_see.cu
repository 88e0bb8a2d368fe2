// Enrichment-enrichment block of S with FP64-class sums (mixed-precision path).
//
// S is ill-conditioned because the enrichments are nearly linearly dependent
// on each other and on the FE functions (Sec. 6.2, Table 1: cond(S) grows to
// 1e9 with the support radius), so the mixed path keeps this block of S free
// of FP32 rounding in its sums while H and the other blocks of S are
// contracted in FP32.
//
// For columns r = (v, alpha) and s = (v', beta) of an element, on one
// (sub)cell with a p^3 tensor rule (Sec. 4 eq. disceig3d, Sec. 5.2),
//   S_rs = sum_q w_q Psi_alpha(x_q) Psi_beta(x_q) phi_v(x_q) phi_v'(x_q).
// The trilinear PU factors give phi_v phi_v' = 1/64 prod_d u_(k_d)(xi_d) with
// u_0 = (1 - x)^2, u_1 = (1 - x)(1 + x), u_2 = (1 + x)^2 and k_d = b_d + b'_d
// the sum of the two vertices' bits along axis d, so every entry of the pair
// (alpha, beta) is one of 27 projections
//   P_ab[kz][ky][kx] = sum_q s_alpha(q) s_beta(q) u_kz(zeta) u_ky(eta) u_kx(xi),
//   s_alpha = sqrt(w) Psi_alpha,
// contracted one axis at a time (3 p^3 + 9 p^2 + 27 p multiply-adds per pair
// and cell, against p^3 per entry for the direct sum):  S_rs = P_ab[k] / 64
// (the 1/64 is carried by the 1D factors, halved per axis).
//
// Arithmetic.  The factors are the FP32 values of the mixed path: s rounded
// once to FP32 from sqrt(w) of the FP32 weight and Psi, the 1D factors
// 1 -+ x from the FP32 reference coordinate.  Every product of two such values is formed
// exactly as an unevaluated FP32 pair (hi + lo, hi = fl(a b), lo = fma(a, b,
// -hi): Dekker's product through the FMA), the u_k are kept exactly that way,
// and every sum is compensated (Knuth's two-sum on the high parts, the low
// parts in FP32), about 2^-48 relative per operation.  So the block is the Gram matrix of the rounded
// basis values to FP64-class accuracy -- no FP32 rounding enters its sums --
// while every instruction runs on the FP32 pipes: GB300 issues FP64 at 1/64
// of the FP32 rate, and the same contraction in plain FP64 took 1.5 times
// as long as the whole FP32 strip.  The pairs are added as FP64 values
// (hi + lo) into the FP64 CSR values with FP64 atomics, both triangles;
// cells of a subdivided element add up there.
#include <algorithm>

#include "pufe_internal.h"

namespace pufe {
namespace {

constexpr int SE_NT = 256;

// an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2)
struct ff {
  float hi, lo;
};

// a b exactly (Dekker's product through the FMA)
__device__ __forceinline__ ff ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// a + b exactly (Knuth's two-sum, no ordering of |a|, |b| needed)
__device__ __forceinline__ ff ff_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// acc + x y for pairs x, y: the product's hi*hi part exactly, its cross terms
// by FMA (the lo*lo term is below 2^-96 relative), the high parts added
// exactly (two-sum) and the low parts summed in FP32, whose rounding is
// ~2^-24 of a ~2^-24 correction; ff_norm folds lo back into hi where a stage
// stores its results (two-sum, exact under cancellation too)
__device__ __forceinline__ ff ff_fma(ff x, ff y, ff acc) {
  const ff p = ff_prod(x.hi, y.hi);
  const float plo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  const ff s = ff_sum(acc.hi, p.hi);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, plo))};
}

__device__ __forceinline__ ff ff_norm(ff a) { return ff_sum(a.hi, a.lo); }

// One CTA per work item: the slot pairs [pb, pe) (alpha-major order) of
// element order[k], (k, pb, pe) = items[3 b .. 3 b + 2].  A (sub)cell's
// sqrt(w) Psi values are staged in shared memory when A p^3 <= stage_f, else
// formed from the table at each use.
template <bool BLOCH>
__global__ void __launch_bounds__(SE_NT) k_see(
    const int32_t *__restrict__ order, const int32_t *__restrict__ items,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const int32_t *__restrict__ partoff, const int32_t *__restrict__ part_p,
    const int32_t *__restrict__ part_q, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap, int pm, int amax,
    int stage_f, int work_ff, double *__restrict__ S, unsigned *err,
    const uint8_t *__restrict__ eshift, PhaseTab ph, double *__restrict__ Si) {
  extern __shared__ float4 sm_see4[];
  const int e = order[items[3 * blockIdx.x]], tid = threadIdx.x;
  const int pb = items[3 * blockIdx.x + 1], pe_ = items[3 * blockIdx.x + 2];
  const int n = (int)(doff[e + 1] - doff[e]), ne = n - 64;
  if (ne <= 0) return;
  const int A = aoff[e + 1] - aoff[e];
  if (A > amax || A > 255) {
    if (tid == 0) atomicOr(err, DEVERR_SHAPE);
    return;
  }
  // shared memory: U [3 axes][u_0, u_1, u_2][pm] pairs | work pairs
  //                | stage [slot][point] floats | scol [slot][vertex] | pairs
  //                | masks [pair][2]
  ff *U = reinterpret_cast<ff *>(sm_see4);
  ff *work = U + 9 * pm;
  float *stg = reinterpret_cast<float *>(work + work_ff);
  int *scol = reinterpret_cast<int *>(stg + stage_f);
  int *pairs = scol + amax * 8;
  int *msk = pairs + amax * (amax + 1) / 2;
  __shared__ double s_phr[8], s_phi[8];
  if (BLOCH && tid < 8) {
    s_phr[tid] = ph.re[tid];
    s_phi[tid] = ph.im[tid];
  }
  const int32_t *ecs = ecol + (doff[e] - 64ll * e);
  for (int o = tid; o < A * 8; o += SE_NT) scol[o] = -1;
  __syncthreads();
  for (int r = tid; r < ne; r += SE_NT) {
    const int c = ecs[r];
    scol[(c >> 3) * 8 + (c & 7)] = r;
  }
  const int npair = A * (A + 1) / 2;
  if (pb < 0 || pe_ > npair || pb >= pe_) {
    if (tid == 0) atomicOr(err, DEVERR_SHAPE);
    return;
  }
  if (tid < A) {   // pairs (alpha, beta), alpha <= beta, alpha-major
    int k = tid * A - tid * (tid - 1) / 2;
    for (int b = tid; b < A; ++b) pairs[k++] = tid | (b << 8);
  }
  __syncthreads();
  // the projections a pair's existing vertex pairs use: kz (3 bits) and
  // (kz, ky) (9 bits) in msk[2 g], (kz, ky, kx) (27 bits) in msk[2 g + 1];
  // the stages skip the others (slots with few vertex columns need few)
  for (int g = pb + tid; g < pe_; g += SE_NT) {
    const int pr = pairs[g], al = pr & 0xff, be = pr >> 8;
    int mz = 0, myz = 0, mxyz = 0;
    for (int i = 0; i < 8; ++i) {
      if (scol[al * 8 + i] < 0) continue;
      for (int j = al == be ? i : 0; j < 8; ++j) {
        if (scol[be * 8 + j] < 0) continue;
        const int kx = (i & 1) + (j & 1), ky = ((i >> 1) & 1) + ((j >> 1) & 1),
                  kz = (i >> 2) + (j >> 2);
        mz |= 1 << kz;
        myz |= 1 << (kz * 3 + ky);
        mxyz |= 1 << ((kz * 3 + ky) * 3 + kx);
      }
    }
    msk[2 * g] = mz | (myz << 3);
    msk[2 * g + 1] = mxyz;
  }
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  const int32_t *m = smap + soff[e];
  const uint8_t *esh = BLOCH ? eshift + doff[e] : nullptr;

  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    const int p = part_p[k], p2 = p * p, p3 = p2 * p, qs = part_q[k];
    const int per = 3 * p2 + 9 * p + 27;   // work pairs of one enrichment pair
    const bool staged = A * p3 <= stage_f;
    if (p > pm || per > work_ff) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    __syncthreads();   // previous cell's users of U, stage and work are done
    for (int o = tid; o < 3 * p; o += SE_NT) {
      const int d = o / p, t = o - d * p;
      const int stride = d == 0 ? 1 : (d == 1 ? p : p2);
      const float4 x4 = qe[qs + t * stride];
      const float x = d == 0 ? x4.x : (d == 1 ? x4.y : x4.z);
      // the PU factors 1/2 (1 -+ x) per axis (exact halving), so the three
      // axes' products carry phi_v phi_v' = 1/64 prod u_k exactly
      const float l0 = 0.5f * __fsub_rn(1.0f, x), l1 = 0.5f * __fadd_rn(1.0f, x);
      U[(d * 3 + 0) * pm + t] = ff_prod(l0, l0);
      U[(d * 3 + 1) * pm + t] = ff_prod(l0, l1);
      U[(d * 3 + 2) * pm + t] = ff_prod(l1, l1);
    }
    // sqrt(w) Psi of a slot at a point of the cell, rounded once to FP32 (w
    // from the point array, Psi from the table [q/8][slot][comp][q%8],
    // component 0)
    auto sval = [&](int slot, int lq) -> float {
      const int q = qs + lq;
      return __fmul_rn(__fsqrt_rn(qe[q].w), pe[((int64_t)(q >> 3) * A + slot) * 32 + (q & 7)]);
    };
    if (staged)
      for (int o = tid; o < A * p3; o += SE_NT) {
        const int s = o / p3, lq = o - s * p3;
        stg[o] = sval(s, lq);
      }
    __syncthreads();
    const int npc = max(1, min(pe_ - pb, work_ff / per));
    for (int c0 = pb; c0 < pe_; c0 += npc) {
      const int nc = min(npc, pe_ - c0);
      ff *T1 = work;                    // [nc][p^2][3]: z outputs
      ff *T2 = T1 + nc * 3 * p2;        // [nc][p][kz][ky]
      ff *P = T2 + nc * 9 * p;          // [nc][kz][ky][kx]
      // z: one thread per (pair, qx, qy) column
      for (int it = tid; it < nc * p2; it += SE_NT) {
        const int g = it / p2, qxy = it - g * p2;
        const int pr = pairs[c0 + g], al = pr & 0xff, be = pr >> 8;
        const int mz = msk[2 * (c0 + g)] & 7;
        ff a0 = {0.0f, 0.0f}, a1 = {0.0f, 0.0f}, a2 = {0.0f, 0.0f};
        for (int qz = 0; qz < p; ++qz) {
          const int lq = qxy + p2 * qz;
          const ff f = staged ? ff_prod(stg[al * p3 + lq], stg[be * p3 + lq])
                              : ff_prod(sval(al, lq), sval(be, lq));
          if (mz & 1) a0 = ff_fma(f, U[6 * pm + qz], a0);
          if (mz & 2) a1 = ff_fma(f, U[7 * pm + qz], a1);
          if (mz & 4) a2 = ff_fma(f, U[8 * pm + qz], a2);
        }
        ff *t1 = T1 + (size_t)it * 3;
        t1[0] = ff_norm(a0);
        t1[1] = ff_norm(a1);
        t1[2] = ff_norm(a2);
      }
      __syncthreads();
      // y: one thread per (pair, qx, kz)
      for (int it = tid; it < nc * p * 3; it += SE_NT) {
        const int g = it / (3 * p), rem = it - g * 3 * p, qx = rem / 3, kz = rem - qx * 3;
        const int my = (msk[2 * (c0 + g)] >> (3 + 3 * kz)) & 7;
        if (!my) continue;
        const ff *t1 = T1 + ((size_t)g * p2 + qx) * 3 + kz;
        ff b0 = {0.0f, 0.0f}, b1 = {0.0f, 0.0f}, b2 = {0.0f, 0.0f};
        for (int qy = 0; qy < p; ++qy) {
          const ff t = t1[qy * p * 3];
          if (my & 1) b0 = ff_fma(t, U[3 * pm + qy], b0);
          if (my & 2) b1 = ff_fma(t, U[4 * pm + qy], b1);
          if (my & 4) b2 = ff_fma(t, U[5 * pm + qy], b2);
        }
        ff *t2 = T2 + ((size_t)g * p + qx) * 9 + kz * 3;
        t2[0] = ff_norm(b0);
        t2[1] = ff_norm(b1);
        t2[2] = ff_norm(b2);
      }
      __syncthreads();
      // x: one thread per (pair, kz, ky)
      for (int it = tid; it < nc * 9; it += SE_NT) {
        const int g = it / 9, j = it - g * 9;
        const int mx = (msk[2 * (c0 + g) + 1] >> (3 * j)) & 7;
        if (!mx) continue;
        const ff *t2 = T2 + (size_t)g * p * 9 + j;
        ff c0v = {0.0f, 0.0f}, c1v = {0.0f, 0.0f}, c2v = {0.0f, 0.0f};
        for (int qx = 0; qx < p; ++qx) {
          const ff t = t2[qx * 9];
          if (mx & 1) c0v = ff_fma(t, U[qx], c0v);
          if (mx & 2) c1v = ff_fma(t, U[pm + qx], c1v);
          if (mx & 4) c2v = ff_fma(t, U[2 * pm + qx], c2v);
        }
        ff *pp = P + g * 27 + j * 3;
        pp[0] = ff_norm(c0v);
        pp[1] = ff_norm(c1v);
        pp[2] = ff_norm(c2v);
      }
      __syncthreads();
      // scatter: one thread per (pair, vertex of alpha, vertex of beta); a
      // pair (alpha, alpha) takes each unordered column pair once
      for (int it = tid; it < nc * 64; it += SE_NT) {
        const int g = it >> 6, i = (it >> 3) & 7, j = it & 7;
        const int pr = pairs[c0 + g], al = pr & 0xff, be = pr >> 8;
        if (al == be && j < i) continue;
        const int r = scol[al * 8 + i], s = scol[be * 8 + j];
        if (r < 0 || s < 0) continue;
        const int kx = (i & 1) + (j & 1), ky = ((i >> 1) & 1) + ((j >> 1) & 1),
                  kz = (i >> 2) + (j >> 2);
        const ff pv = P[g * 27 + (kz * 3 + ky) * 3 + kx];
        const double v = (double)pv.hi + (double)pv.lo;
        const int s_rs = m[(64 + r) * n + 64 + s], s_sr = m[(64 + s) * n + 64 + r];
        if (BLOCH) {   // (r, s) with conj(ph_r) ph_s, (s, r) with its conjugate
          const int a = esh[64 + r], b = esh[64 + s];
          const double pr_ = s_phr[a] * s_phr[b] + s_phi[a] * s_phi[b];
          const double pi_ = s_phr[a] * s_phi[b] - s_phi[a] * s_phr[b];
          atomicAdd(S + s_rs, v * pr_);
          atomicAdd(Si + s_rs, v * pi_);
          if (r != s) {
            atomicAdd(S + s_sr, v * pr_);
            atomicAdd(Si + s_sr, -v * pi_);
          }
        } else {
          atomicAdd(S + s_rs, v);
          if (r != s) atomicAdd(S + s_sr, v);
        }
      }
      __syncthreads();   // P and the work area are reused by the next chunk
    }
  }
}


// Gram form, for elements whose (sub)cells hold more Psi values than the
// projection kernel's stage: S_rs = sum_q c_r(q) c_s(q) over the element's
// points with the column values c_r = s_alpha phi_v as unevaluated pairs:
// s_alpha = fl(sqrt(w) Psi_alpha) as above, phi_v = l_x l_y l_z with the exact
// halved linears l = (1 -+ xi) / 2 of the vertex's bits (the same factors as
// the projection form), each product of a pair and an FP32 value kept as a
// pair (~2^-48), the pair products and their sums as in ff_fma.  Work item
// b: (order index, row tile, column tile, first point, end point) =
// items[5 b .. 5 b + 4]; tiles of 16 TB enrichment columns, each thread a
// TB x TB block of (r, s) pairs; points in chunks of GK, the chunk's column
// values staged in shared memory (hi and lo parts apart, point-major).  The
// lower triangle (r >= s) goes into both triangles of S; the point ranges of
// an element meet in the FP64 atomics.
constexpr int GK = 32;

template <bool BLOCH, int TB>
__global__ void __launch_bounds__(SE_NT) k_see_gram(
    const int32_t *__restrict__ order, const int32_t *__restrict__ items,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ ecol,
    const int32_t *__restrict__ aoff, const int64_t *__restrict__ toff32,
    const float *__restrict__ psi, const int64_t *__restrict__ soff,
    const int32_t *__restrict__ smap, double *__restrict__ S, unsigned *err,
    const uint8_t *__restrict__ eshift, PhaseTab ph, double *__restrict__ Si) {
  constexpr int T = 16 * TB;   // columns per tile
  __shared__ float rh[GK][T], rl[GK][T], ch[GK][T], cl[GK][T];
  __shared__ double s_phr[8], s_phi[8];
  const int tid = threadIdx.x;
  const int *it5 = items + 5 * blockIdx.x;
  const int e = order[it5[0]], rt = it5[1], ct = it5[2], qa = it5[3], qb = it5[4];
  const int n = (int)(doff[e + 1] - doff[e]), ne = n - 64;
  const int A = aoff[e + 1] - aoff[e];
  if (ne <= 0 || ct > rt || (rt + 1) * T > ((ne + T - 1) / T) * T || qa < 0 || qb <= qa ||
      (int64_t)qb > qpoff[e + 1] - qpoff[e]) {
    if (tid == 0) atomicOr(err, DEVERR_SHAPE);
    return;
  }
  if (BLOCH && tid < 8) {
    s_phr[tid] = ph.re[tid];
    s_phi[tid] = ph.im[tid];
  }
  const int32_t *ecs = ecol + (doff[e] - 64ll * e);
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  const int r0 = rt * T, c0 = ct * T;
  const int ti = tid >> 4, tj = tid & 15;
  ff acc[TB][TB];
#pragma unroll
  for (int a = 0; a < TB; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) acc[a][b] = {0.0f, 0.0f};
  // c_r at point q of the element (zero past the element's columns)
  auto colval = [&](int r, int q) -> ff {
    if (r >= ne) return {0.0f, 0.0f};
    const int code = ecs[r], lv = code & 7, slot = code >> 3;
    if (slot >= A) return {0.0f, 0.0f};
    const float4 x4 = qe[q];
    const float xs[3] = {x4.x, x4.y, x4.z};
    float l[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      l[d] = ((lv >> d) & 1) ? 0.5f * __fadd_rn(1.0f, xs[d]) : 0.5f * __fsub_rn(1.0f, xs[d]);
    const float sv = __fmul_rn(__fsqrt_rn(x4.w), pe[((int64_t)(q >> 3) * A + slot) * 32 + (q & 7)]);
    ff t = ff_prod(l[0], l[1]);                        // exact
    ff u = ff_prod(t.hi, l[2]);
    u.lo = __fmaf_rn(t.lo, l[2], u.lo);                // phi_v as a pair
    ff c = ff_prod(u.hi, sv);
    c.lo = __fmaf_rn(u.lo, sv, c.lo);                  // s phi_v as a pair
    return ff_norm(c);
  };
  for (int q0 = qa; q0 < qb; q0 += GK) {
    __syncthreads();   // the previous chunk's readers are done
    for (int o = tid; o < GK * T; o += SE_NT) {
      const int kq = o / T, j = o - kq * T, q = q0 + kq;
      ff vr = {0.0f, 0.0f}, vc = {0.0f, 0.0f};
      if (q < qb) {
        vr = colval(r0 + j, q);
        vc = (ct == rt) ? vr : colval(c0 + j, q);
      }
      rh[kq][j] = vr.hi;
      rl[kq][j] = vr.lo;
      ch[kq][j] = vc.hi;
      cl[kq][j] = vc.lo;
    }
    __syncthreads();
    const int nk = min(GK, qb - q0);
    for (int kq = 0; kq < nk; ++kq) {
      ff xr[TB], xc[TB];
#pragma unroll
      for (int a = 0; a < TB; ++a) xr[a] = {rh[kq][ti * TB + a], rl[kq][ti * TB + a]};
#pragma unroll
      for (int b = 0; b < TB; ++b) xc[b] = {ch[kq][tj * TB + b], cl[kq][tj * TB + b]};
#pragma unroll
      for (int a = 0; a < TB; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) acc[a][b] = ff_fma(xr[a], xc[b], acc[a][b]);
    }
  }
  // the lower triangle into both triangles of S
  const int32_t *m = smap + soff[e];
  const uint8_t *esh = BLOCH ? eshift + doff[e] : nullptr;
#pragma unroll
  for (int a = 0; a < TB; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) {
      const int r = r0 + ti * TB + a, sc = c0 + tj * TB + b;
      if (r >= ne || sc >= ne || sc > r) continue;
      const ff pv = ff_norm(acc[a][b]);
      const double v = (double)pv.hi + (double)pv.lo;
      const int s_rs = m[(64 + r) * n + 64 + sc], s_sr = m[(64 + sc) * n + 64 + r];
      if (BLOCH) {   // (r, s) with conj(ph_r) ph_s, (s, r) with its conjugate
        const int ca = esh[64 + r], cb = esh[64 + sc];
        const double pr_ = s_phr[ca] * s_phr[cb] + s_phi[ca] * s_phi[cb];
        const double pi_ = s_phr[ca] * s_phi[cb] - s_phi[ca] * s_phr[cb];
        atomicAdd(S + s_rs, v * pr_);
        atomicAdd(Si + s_rs, v * pi_);
        if (r != sc) {
          atomicAdd(S + s_sr, v * pr_);
          atomicAdd(Si + s_sr, -v * pi_);
        }
      } else {
        atomicAdd(S + s_rs, v);
        if (r != sc) atomicAdd(S + s_sr, v);
      }
    }
}

}  // namespace

// Work area of the projection form (FP32 pairs): the stage outputs of a chunk
// of slot pairs.
static constexpr int SEE_WORK_FF = 2048;

pufe_status launch_see(pufe_ctx *ctx, const PhaseTab *ph, double *S, double *Si, cudaStream_t st) {
  auto &D = ctx->d;
  // the Gram form first (the elements too large for the stage: the heaviest
  // items), 32- and 64-column tiles
  auto gram = [&](auto k32, auto k64, const uint8_t *esh, PhaseTab tab, double *si) -> pufe_status {
    if (ctx->n_gitems32 > 0) {
      k32<<<(unsigned)ctx->n_gitems32, SE_NT, 0, st>>>(D.order, D.gitems32, D.qpoff, D.qdat,
                                                        D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
                                                        D.soff, D.smap, S, D.err, esh, tab, si);
      PUFE_CUDA_TRY(cudaGetLastError());
    }
    if (ctx->n_gitems64 > 0) {
      k64<<<(unsigned)ctx->n_gitems64, SE_NT, 0, st>>>(D.order, D.gitems64, D.qpoff, D.qdat,
                                                        D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
                                                        D.soff, D.smap, S, D.err, esh, tab, si);
      PUFE_CUDA_TRY(cudaGetLastError());
    }
    return PUFE_OK;
  };
  const pufe_status eg = ph ? gram(k_see_gram<true, 2>, k_see_gram<true, 4>, D.eshift, *ph, Si)
                            : gram(k_see_gram<false, 2>, k_see_gram<false, 4>, nullptr,
                                   PhaseTab{}, nullptr);
  if (eg != PUFE_OK) return eg;
  if (ctx->n_sitems <= 0) return PUFE_OK;
  const int pm = std::max(1, ctx->max_part_p);
  const int amax = std::max(1, ctx->max_alpha);
  if (amax > 255) return fail(PUFE_EINVAL, "more than 255 enrichments on one element");
  const int per_max = 3 * pm * pm + 9 * pm + 27;
  const int work = std::max(SEE_WORK_FF, per_max);
  // the stage is sized for the largest cell that fits the budget
  int stage = 0;
  for (int64_t e = 0; e < ctx->nelem; ++e)
    if (ctx->see_stage[e] <= SEE_STAGE_MAX_F) stage = std::max(stage, (int)ctx->see_stage[e]);
  const size_t ints = (size_t)amax * 8 + (size_t)3 * amax * (amax + 1) / 2;
  const size_t sm = ((size_t)9 * pm + work) * sizeof(ff) + (size_t)stage * sizeof(float) +
                    ints * sizeof(int);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "E-E overlap kernel: shared memory above 227 KB");
  auto go = [&](auto kern, const uint8_t *esh, PhaseTab tab, double *si) -> pufe_status {
    PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<(unsigned)ctx->n_sitems, SE_NT, sm, st>>>(
        D.order, D.sitems, D.qpoff, D.qdat, D.partoff, D.part_p, D.part_q, D.doff, D.ecol,
        D.aoff, D.toff32, D.psi32, D.soff, D.smap, pm, amax, stage, work, S, D.err, esh, tab, si);
    PUFE_CUDA_TRY(cudaGetLastError());
    return PUFE_OK;
  };
  if (ph) return go(k_see<true>, D.eshift, *ph, Si);
  return go(k_see<false>, nullptr, PhaseTab{}, nullptr);
}

}  // namespace pufe
