// FE-FE block of H_V = int phi_i V phi_j by sum factorization (mixed path).
//
// On a tensor-product (sub)cell rule with points q = (qx, qy, qz), the 64
// tricubic functions are products L_a(x) L_b(y) L_c(z), so
//   M[(a,b,c),(a',b',c')] = sum_q w_q V_q L_a L_a' L_b L_b' L_c L_c'
// contracts one axis at a time: first z for every (qx, qy), then y, then x.
// The integrand is symmetric in each axis pair separately, so M has only
// 10 x 10 x 10 distinct values (unordered pairs per axis).  Cost per p^3 cell:
// 10 p^3 + 100 p^2 + 1000 p multiply-adds, against 2080 p^3 for the direct
// element contraction.  (Sec. 4 eq. disceig3d, local potential term; the rule
// is the element's shared rule of Sec. 5.2.)
//
// H starts at zero; each element adds the constant 64 x 64 kinetic block of
// the tricubic functions (the same on every element of the cubic mesh, exact
// for rules with >= 4 points per axis, precomputed in FP64) plus its block of
// M through the scatter map.  The enrichment strip kernel adds the rest.
#include <algorithm>

#include "pufe_internal.h"

namespace pufe {
namespace {

constexpr int SF_NT = 128;
constexpr int SF_PMAX = 16;

__device__ __forceinline__ int pidx(int a, int b) {  // unordered pair -> 0..9
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo * 4 - (lo * (lo - 1)) / 2 + (hi - lo);
}

__device__ __forceinline__ void lag3(float t, float L[4]) {
  const float a = t + 1.0f, b = t + (1.0f / 3.0f), c = t - (1.0f / 3.0f), d = t - 1.0f;
  L[0] = -0.5625f * b * c * d;
  L[1] = 1.6875f * a * c * d;
  L[2] = -1.6875f * a * b * d;
  L[3] = 0.5625f * a * b * c;
}

// BLOCH (Sec. 4, eqs. bloch, strong): entry (i, j) goes into H(k) and S(k)
// with the phase conj(exp(i k.R_i)) exp(i k.R_j) of the columns' lattice
// shifts, the constant overlap block included (S(k) has no k-independent part).
template <bool BLOCH>
__global__ void __launch_bounds__(SF_NT) k_fefe_sumfac(
    const int64_t *__restrict__ qoff, const double *__restrict__ w, const double *__restrict__ V,
    const double *__restrict__ xi_all, const int32_t *__restrict__ partoff,
    const int32_t *__restrict__ part_p, const int32_t *__restrict__ part_q,
    const int64_t *__restrict__ doff, const int64_t *__restrict__ soff,
    const int32_t *__restrict__ smap, const double *__restrict__ Tfe, double *__restrict__ H,
    unsigned *err, const double *__restrict__ Sfe, const uint8_t *__restrict__ eshift,
    PhaseTab ph, int what, double *__restrict__ Hi, double *__restrict__ S,
    double *__restrict__ Si) {
  __shared__ float Wq[SF_PMAX * SF_PMAX * SF_PMAX];
  __shared__ float P[3][10][SF_PMAX];          // pair products per axis
  __shared__ float G1[SF_PMAX * SF_PMAX * 10];  // [qx + p qy][cc]
  __shared__ float G2[SF_PMAX * 100];           // [qx][bb * 10 + cc]
  __shared__ float M[1000];
  const int e = blockIdx.x, tid = threadIdx.x;
  for (int o = tid; o < 1000; o += SF_NT) M[o] = 0.0f;
  for (int k = partoff[e]; V != nullptr && k < partoff[e + 1]; ++k) {
    const int p = part_p[k];
    if (p > SF_PMAX) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    const int64_t qs = qoff[e] + part_q[k];
    const int p2 = p * p, p3 = p2 * p;
    __syncthreads();
    bool bad = false;
    for (int q = tid; q < p3; q += SF_NT) {
      const double v = V[qs + q];
      bad |= !isfinite(v);
      Wq[q] = (float)(w[qs + q] * v);
    }
    if (bad) atomicOr(err, DEVERR_NONFINITE);
    for (int o = tid; o < 3 * p; o += SF_NT) {
      const int d = o / p, t = o - d * p;
      const int stride = d == 0 ? 1 : (d == 1 ? p : p2);
      float L[4];
      lag3((float)xi_all[3 * (qs + (int64_t)t * stride) + d], L);
      int c = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b) P[d][c++][t] = L[a] * L[b];
    }
    __syncthreads();
    for (int o = tid; o < p2 * 10; o += SF_NT) {  // contract z
      const int qxy = o / 10, cc = o - qxy * 10;
      float s = 0.0f;
      for (int qz = 0; qz < p; ++qz) s = fmaf(Wq[qxy + p2 * qz], P[2][cc][qz], s);
      G1[o] = s;
    }
    __syncthreads();
    for (int o = tid; o < p * 100; o += SF_NT) {  // contract y
      const int qx = o / 100, r = o - qx * 100, bb = r / 10, cc = r - bb * 10;
      float s = 0.0f;
      for (int qy = 0; qy < p; ++qy) s = fmaf(P[1][bb][qy], G1[(qx + p * qy) * 10 + cc], s);
      G2[o] = s;
    }
    __syncthreads();
    for (int o = tid; o < 1000; o += SF_NT) {  // contract x
      const int aa = o / 100, r = o - aa * 100;
      float s = 0.0f;
      for (int qx = 0; qx < p; ++qx) s = fmaf(P[0][aa][qx], G2[qx * 100 + r], s);
      M[o] += s;
    }
  }
  __syncthreads();
  // add the 64 x 64 block into H through the scatter map: thread pairs
  // (i, j) run along j, so consecutive lanes hit neighbouring CSR columns
  const int n = (int)(doff[e + 1] - doff[e]);
  const int32_t *m = smap + soff[e];
  for (int o = tid; o < 64 * 64; o += SF_NT) {
    const int i = o >> 6, j = o & 63;
    const float v = M[pidx(i & 3, j & 3) * 100 + pidx((i >> 2) & 3, (j >> 2) & 3) * 10 +
                      pidx(i >> 4, j >> 4)];
    const int slot = m[i * n + j];
    if (!BLOCH) {
      atomicAdd(H + slot, __ldg(Tfe + o) + (double)v);
    } else {
      const int ci = eshift[doff[e] + i], cj = eshift[doff[e] + j];
      const double pr = ph.re[ci] * ph.re[cj] + ph.im[ci] * ph.im[cj];
      const double pi = ph.re[ci] * ph.im[cj] - ph.im[ci] * ph.re[cj];
      if (what & PUFE_WANT_H) {
        const double hv = __ldg(Tfe + o) + (double)v;
        atomicAdd(H + slot, hv * pr);
        atomicAdd(Hi + slot, hv * pi);
      }
      if (what & PUFE_WANT_S) {
        const double sv = __ldg(Sfe + o);
        atomicAdd(S + slot, sv * pr);
        atomicAdd(Si + slot, sv * pi);
      }
    }
  }
}

// FE-FE part of the adjoint of V -> H on a tensor-product (sub)cell:
//   f(q) = sum_{(abc),(a'b'c')} L_a L_a' L_b L_b' L_c L_c' Hbar[(abc),(a'b'c')]
// (Hbar restricted to the element's 64 FE columns, general, not symmetric),
// contracted axis by axis: 4096 p + 256 p^2 + 16 p^3 multiply-adds per cell,
// then Vbar_q = w_q f(q) is stored (the strip kernel adds the enrichment part).
template <bool BLOCH>
__global__ void __launch_bounds__(SF_NT) k_adjoint_fefe(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const double *__restrict__ w, const double *__restrict__ xi_all,
    const int32_t *__restrict__ partoff, const int32_t *__restrict__ part_p,
    const int32_t *__restrict__ part_q, const int64_t *__restrict__ doff,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap,
    const double *__restrict__ Hbar, int pm, double *__restrict__ Vbar, unsigned *err,
    BlochCot bc) {
  // dynamic shared memory, sized for the largest per-axis count pm:
  // Hs[64][64], L1[3][4][pm], G1[256 pm] = [(a,b),(a',b')][qz],
  // G2[16 pm^2] = [(a,a')][qy + p qz]
  extern __shared__ float sm_adj[];
  float *Hs = sm_adj, *L1 = Hs + 4096, *G1 = L1 + 12 * pm, *G2 = G1 + 256 * pm;
  const int e = order[blockIdx.x], tid = threadIdx.x;
  const int n = (int)(doff[e + 1] - doff[e]);
  const int32_t *m = smap + soff[e];
  // gather with eight independent (map, value) load chains in flight per thread
  for (int o0 = tid; o0 < 4096; o0 += 8 * SF_NT) {
    int s1[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int o = o0 + u * SF_NT;
      s1[u] = o < 4096 ? m[(o >> 6) * n + (o & 63)] : 0;
    }
    double h[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) h[u] = o0 + u * SF_NT < 4096 ? Hbar[s1[u]] : 0.0;
    if (BLOCH) {   // at a wavevector: the phased real part (columns' shift codes)
      double hi[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) hi[u] = o0 + u * SF_NT < 4096 ? bc.Hi[s1[u]] : 0.0;
      const uint8_t *esh = bc.eshift + doff[e];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int o = o0 + u * SF_NT;
        if (o < 4096) h[u] = cot_entry(h[u], hi[u], esh[o >> 6], esh[o & 63], bc.ph);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (o0 + u * SF_NT < 4096) Hs[o0 + u * SF_NT] = (float)h[u];
  }
  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    const int p = part_p[k];
    if (p > pm) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    const int64_t qs = qoff[e] + part_q[k];
    const int p2 = p * p, p3 = p2 * p;
    __syncthreads();
    for (int o = tid; o < 3 * p; o += SF_NT) {
      const int d = o / p, t = o - d * p;
      const int stride = d == 0 ? 1 : (d == 1 ? p : p2);
      float L[4];
      lag3((float)xi_all[3 * (qs + (int64_t)t * stride) + d], L);
      for (int a = 0; a < 4; ++a) L1[(d * 4 + a) * pm + t] = L[a];
    }
    __syncthreads();
    // contract (c, c') for each qz: G1[(a,b),(a',b')][qz]
    for (int o = tid; o < 256 * p; o += SF_NT) {
      const int pr = o / p, qz = o - pr * p;
      const int ab = pr >> 4, apbp = pr & 15;   // (a + 4b), (a' + 4b')
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int cp = 0; cp < 4; ++cp)
          s = fmaf(L1[(8 + c) * pm + qz] * L1[(8 + cp) * pm + qz], Hs[(ab + 16 * c) * 64 + apbp + 16 * cp], s);
      G1[o] = s;
    }
    __syncthreads();
    // contract (b, b') for each (qy, qz): G2[(a,a')][qy + p qz]
    for (int o = tid; o < 16 * p2; o += SF_NT) {
      const int aa = o / p2, r = o - aa * p2, qy = r % p, qz = r / p;
      const int a = aa >> 2, ap = aa & 3;
      float s = 0.0f;
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int bp = 0; bp < 4; ++bp)
          s = fmaf(L1[(4 + b) * pm + qy] * L1[(4 + bp) * pm + qy], G1[((a + 4 * b) * 16 + ap + 4 * bp) * p + qz], s);
      G2[o] = s;
    }
    __syncthreads();
    // contract (a, a') for each point, store w_q f(q)
    for (int q = tid; q < p3; q += SF_NT) {
      const int qx = q % p, r = q / p;
      float s = 0.0f;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int ap = 0; ap < 4; ++ap)
          s = fmaf(L1[a * pm + qx] * L1[ap * pm + qx], G2[(a * 4 + ap) * p2 + r], s);
      Vbar[qs + q] = w[qs + q] * (double)s;
    }
  }
}

}  // namespace

// Every element adds its kinetic FE-FE block and the FE-FE block of H_V into
// H (which the caller has zeroed); V == NULL means V = 0.
pufe_status launch_fefe(pufe_ctx *ctx, const double *V, double *H, cudaStream_t st) {
  auto &D = ctx->d;
  if (ctx->max_part_p > SF_PMAX) return fail(PUFE_EINVAL, "rule with more than 16 points per axis");
  if (!D.Tfe) return fail(PUFE_ESTATE, "no exact FE-FE blocks (a rule has < 4 points per axis)");
  k_fefe_sumfac<false><<<(unsigned)ctx->nelem, SF_NT, 0, st>>>(
      D.qoff, D.w, V, D.xi, D.partoff, D.part_p, D.part_q, D.doff, D.soff, D.smap, D.Tfe, H, D.err,
      nullptr, nullptr, PhaseTab{}, PUFE_WANT_H, nullptr, nullptr, nullptr);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

// Bloch form: the FE-FE blocks of H(k) (if wanted; V == NULL means V = 0) and
// S(k) (if wanted) with the column phases, into zeroed outputs
pufe_status launch_fefe_bloch(pufe_ctx *ctx, const PhaseTab &ph, const double *V, int what,
                              double *H, double *Hi, double *S, double *Si, cudaStream_t st) {
  auto &D = ctx->d;
  if (ctx->max_part_p > SF_PMAX) return fail(PUFE_EINVAL, "rule with more than 16 points per axis");
  if (!D.Tfe || !D.Sfe) return fail(PUFE_ESTATE, "no exact FE-FE blocks (a rule has < 4 points per axis)");
  k_fefe_sumfac<true><<<(unsigned)ctx->nelem, SF_NT, 0, st>>>(
      D.qoff, D.w, (what & PUFE_WANT_H) ? V : nullptr, D.xi, D.partoff, D.part_p, D.part_q,
      D.doff, D.soff, D.smap, D.Tfe, H, D.err, D.Sfe, D.eshift, ph, what, Hi, S, Si);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

}  // namespace pufe

namespace pufe {
// Vbar = w_q (FE part of b^T Hbar b) for elements order[first .. first+count)
pufe_status launch_adjoint_fefe(pufe_ctx *ctx, const double *Hbar, double *Vbar, int first,
                                int count, cudaStream_t st, const BlochCot &bc) {
  auto &D = ctx->d;
  if (ctx->max_part_p > SF_PMAX) return fail(PUFE_EINVAL, "rule with more than 16 points per axis");
  if (count <= 0) return PUFE_OK;
  const int pm = std::max(1, ctx->max_part_p);
  const size_t sm = (size_t)(4096 + 12 * pm + 256 * pm + 16 * pm * pm) * sizeof(float);
  auto kern = bc.Hi ? k_adjoint_fefe<true> : k_adjoint_fefe<false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<(unsigned)count, SF_NT, sm, st>>>(D.order + first, D.qoff, D.w, D.xi, D.partoff, D.part_p,
                                           D.part_q, D.doff, D.soff, D.smap, Hbar, pm, Vbar, D.err,
                                           bc);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}
}  // namespace pufe
