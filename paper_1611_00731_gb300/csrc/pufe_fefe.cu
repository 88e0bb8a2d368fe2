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
// k_h_init then writes every CSR value of H: the precomputed constant kinetic
// FE-FE sum T0 plus, for FE-FE slots, the sum of M over the (at most 8)
// elements that contain both nodes.  Enrichment slots start at T0 = 0; the
// tensor-core strip kernel adds their values afterwards.
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

__global__ void __launch_bounds__(SF_NT) k_fefe_sumfac(
    const int64_t *__restrict__ qoff, const double *__restrict__ w, const double *__restrict__ V,
    const double *__restrict__ xi_all, const int32_t *__restrict__ partoff,
    const int32_t *__restrict__ part_p, const int32_t *__restrict__ part_q,
    float *__restrict__ mfe, unsigned *err) {
  __shared__ float Wq[SF_PMAX * SF_PMAX * SF_PMAX];
  __shared__ float P[3][10][SF_PMAX];          // pair products per axis
  __shared__ float G1[SF_PMAX * SF_PMAX * 10];  // [qx + p qy][cc]
  __shared__ float G2[SF_PMAX * 100];           // [qx][bb * 10 + cc]
  __shared__ float M[1000];
  const int e = blockIdx.x, tid = threadIdx.x;
  for (int o = tid; o < 1000; o += SF_NT) M[o] = 0.0f;
  for (int k = partoff[e]; k < partoff[e + 1]; ++k) {
    const int p = part_p[k];
    if (p > SF_PMAX) {
      if (tid == 0) atomicOr(err, DEVERR_SHAPE);
      return;
    }
    const int64_t qs = qoff[e] + part_q[k];
    const int p2 = p * p, p3 = p2 * p;
    __syncthreads();
    for (int q = tid; q < p3; q += SF_NT) Wq[q] = (float)(w[qs + q] * V[qs + q]);
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
  for (int o = tid; o < 1000; o += SF_NT) mfe[(int64_t)e * 1000 + o] = M[o];
}

// the (element index, local node index) pairs of a node coordinate along one
// axis (a vertex node belongs to two elements; with one element per axis the
// node appears twice in it)
__device__ __forceinline__ int node_elems(int x, int nel, int ex[2], int a[2]) {
  ex[0] = x / 3;
  a[0] = x - 3 * ex[0];
  if (a[0] != 0) return 1;
  ex[1] = (ex[0] - 1 + nel) % nel;
  a[1] = 3;
  return 2;
}

__device__ __forceinline__ int axis_matches(int x1, int x2, int nel, int ex[4], int pr[4]) {
  int e1[2], a1[2], e2[2], a2[2];
  const int c1 = node_elems(x1, nel, e1, a1), c2 = node_elems(x2, nel, e2, a2);
  int c = 0;
  for (int i = 0; i < c1; ++i)
    for (int j = 0; j < c2; ++j)
      if (e1[i] == e2[j]) {
        ex[c] = e1[i];
        pr[c] = pidx(a1[i], a2[j]);
        ++c;
      }
  return c;
}

__global__ void k_h_init(int64_t nrow, int64_t n_fe, int nx, int ny, int nz,
                         const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                         const double *__restrict__ T0, const float *__restrict__ mfe,
                         double *__restrict__ H) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nrow) return;
  const int mx = 3 * nx, my = 3 * ny;
  const bool fe_row = row < n_fe;
  const int x1 = (int)(row % mx), y1 = (int)((row / mx) % my), z1 = (int)(row / ((int64_t)mx * my));
  for (int64_t k = rowptr[row] + lane; k < rowptr[row + 1]; k += 32) {
    double v = T0[k];
    const int g2 = col[k];
    if (fe_row && g2 < n_fe) {
      const int x2 = g2 % mx, y2 = (g2 / mx) % my, z2 = g2 / (mx * my);
      int exs[4], pxs[4], eys[4], pys[4], ezs[4], pzs[4];
      const int cx = axis_matches(x1, x2, nx, exs, pxs);
      const int cy = axis_matches(y1, y2, ny, eys, pys);
      const int cz = axis_matches(z1, z2, nz, ezs, pzs);
      for (int i = 0; i < cx; ++i)
        for (int j = 0; j < cy; ++j)
          for (int l = 0; l < cz; ++l) {
            const int64_t e = exs[i] + (int64_t)nx * (eys[j] + (int64_t)ny * ezs[l]);
            v += (double)mfe[e * 1000 + pxs[i] * 100 + pys[j] * 10 + pzs[l]];
          }
    }
    H[k] = v;
  }
}

}  // namespace

// H = T0 + (FE-FE block of H_V) on every CSR slot; V == NULL means V = 0.
pufe_status launch_fefe(pufe_ctx *ctx, const double *V, double *H, cudaStream_t st) {
  auto &D = ctx->d;
  if (ctx->max_part_p > SF_PMAX) return fail(PUFE_EINVAL, "rule with more than 16 points per axis");
  if (V) {
    k_fefe_sumfac<<<(unsigned)ctx->nelem, SF_NT, 0, st>>>(D.qoff, D.w, V, D.xi, D.partoff, D.part_p,
                                                          D.part_q, D.mfe, D.err);
    PUFE_CUDA_TRY(cudaGetLastError());
  } else {
    PUFE_CUDA_TRY(cudaMemsetAsync(D.mfe, 0, (size_t)ctx->nelem * 1000 * sizeof(float), st));
  }
  const int64_t threads = ctx->n_dof * 32;
  k_h_init<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      ctx->n_dof, ctx->n_fe, ctx->nel[0], ctx->nel[1], ctx->nel[2], D.rowptr, D.col, D.T0, D.mfe, H);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

}  // namespace pufe
