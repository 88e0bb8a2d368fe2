// Mixed-precision (PUFE_TF32X3) kernels of the PUFE hot path on sm_103a.
//
//   K0' FP32 tabulation of Psi and grad Psi (Sec. 5.1).
//   K1+K2+K3 element contraction on the 5th-generation tensor cores
//       (tcgen05.mma kind::tf32, accumulators in tensor memory) with every
//       operand split as x = hi + lo (both TF32) and the product formed as
//       hi*hi + hi*lo + lo*hi, followed by an FP64 scatter into CSR.
//   K4' FP32 density and K5' FP32 adjoint on the CUDA cores.
//
// Structure used (exact, Sec. 4 eq. disceig3d with the rule of Sec. 5.2):
// the FE-FE blocks of T = 1/2 int grad phi . grad phi and of S are polynomial
// integrands of degree <= 6 per axis, integrated exactly by every rule with
// p >= 4 points per axis on each (sub)cell, so they are the same constant
// 64x64 matrices on every element.  Their global sum is precomputed in FP64
// at build time; the tensor cores compute H_V = B^T W_V B for all column
// pairs and T, S only for the pairs that involve an enrichment column.
#include <math.h>

#include "pufe_internal.h"

namespace pufe {

namespace {

constexpr int TC_NT = 256;          // 8 warps: all fill, warp 0 issues, all drain
constexpr int NTILES = 10;          // Y0,Y1,Y2,Z,ZV x (hi, lo)
constexpr int STAGE_BYTES = 81920;  // 10 tiles x (R x KC) fp32 with R x KC = 2048
constexpr int NSTAGE = 2;
constexpr uint64_t WAIT_NS = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for completion `parity` of an mbarrier, giving up after WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (globaltimer() - t0 > WAIT_NS) return false;
  }
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes; `lbo` = byte distance
// between core matrices adjacent along K, `sbo` = along M/N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, swizzle none
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void set_err(unsigned *err, unsigned bit) { atomicOr(err, bit); }

// 1D bulk copy global -> shared (TMA engine), completion counted in bytes on
// an mbarrier.  Sizes are multiples of 16 bytes; addresses 16-byte aligned.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One image of Psi~ h in FP32 (see orbital_accumulate for the formulas).
__device__ __forceinline__ void orb_acc_f(const OrbitalF &o, float dx, float dy, float dz,
                                          float &psi, float g[3]) {
  const float r2 = dx * dx + dy * dy + dz * dz;
  if (r2 >= o.rc * o.rc) return;
  const float r = sqrtf(r2);
  const float x = r * o.inv_rc;
  const float x3 = x * x * x;
  const float hc = 1.0f + x3 * x * (-35.0f + x * (84.0f + x * (-70.0f + 20.0f * x)));
  const float omx = 1.0f - x;
  const float dh = -140.0f * x3 * omx * omx * omx * o.inv_rc;
  const int k = o.n - 1 - o.l;
  const float ez = o.norm * expf(-o.zeta * r);
  float rk = 1.0f, rkm1 = 0.0f;
  for (int i = 0; i < k; ++i) {
    rkm1 = rk;
    rk *= r;
  }
  const float f = ez * rk * hc;
  const float df = ez * ((float)k * rkm1 * hc - o.zeta * rk * hc + rk * dh);
  float gs[3];
  const float S = solid_harmonic<float>(o.l, o.m, dx, dy, dz, gs);
  psi += f * S;
  const float sr = (r > 1e-14f) ? df * S / r : 0.0f;
  g[0] += sr * dx + f * gs[0];
  g[1] += sr * dy + f * gs[1];
  g[2] += sr * dz + f * gs[2];
}

// cubic Lagrange values/slopes in FP32
__device__ __forceinline__ void lagrange3f(float t, float L[4], float dL[4]) {
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

// ---------------------------------------------------------------------------
// K0' (FP32).  Table layout per element: 32-float blocks
//   psi32[4*toff32[e] + ((q/8) * A + slot) * 32 + comp * 8 + q%8]
// so that any run of 8-point blocks is one contiguous, 16-byte aligned span.
// The displacement from the atom is formed as (origin_hi + local) + origin_lo
// with the element-origin displacement precomputed in FP64 and split into two
// floats, so it keeps FP32 accuracy even next to the nucleus.
// ---------------------------------------------------------------------------
__global__ void k_tabulate_f32(const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
                               const int32_t *__restrict__ aoff, const int32_t *__restrict__ alist,
                               const int64_t *__restrict__ toff32, const OrbitalF *__restrict__ orbf,
                               const float *__restrict__ eorig, float ax, float ay, float az,
                               float hx, float hy, float hz, float *__restrict__ psi) {
  const int64_t e = blockIdx.x;
  const int Qp = (int)(qpoff[e + 1] - qpoff[e]);
  const int A = aoff[e + 1] - aoff[e];
  const float av[3] = {ax, ay, az};
  const float inv_a[3] = {1.0f / ax, 1.0f / ay, 1.0f / az};
  const float hh[3] = {0.5f * hx, 0.5f * hy, 0.5f * hz};
  float *out = psi + 4 * toff32[e];
  for (int idx = threadIdx.x; idx < Qp * A; idx += blockDim.x) {
    const int slot = idx / Qp, q = idx - slot * Qp;
    const OrbitalF o = orbf[alist[aoff[e] + slot]];
    const float *eo = eorig + 8 * (int64_t)(aoff[e] + slot);
    const float4 xq = qdat[qpoff[e] + q];
    const float xi[3] = {xq.x, xq.y, xq.z};
    float d[3];
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      d[k] = (eo[k] + (xi[k] + 1.0f) * hh[k]) + eo[3 + k];
      const float rcw = o.rc * 1.0001f;
      lo[k] = (int)ceilf((-rcw - d[k]) * inv_a[k]);
      hi[k] = (int)floorf((rcw - d[k]) * inv_a[k]);
    }
    float v = 0.0f, g[3] = {0.0f, 0.0f, 0.0f};
    for (int i = lo[0]; i <= hi[0]; ++i)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int k = lo[2]; k <= hi[2]; ++k)
          orb_acc_f(o, d[0] + i * av[0], d[1] + j * av[1], d[2] + k * av[2], v, g);
    float *dst = out + ((int64_t)(q >> 3) * A + slot) * 32 + (q & 7);
    dst[0] = v;
    dst[8] = g[0];
    dst[16] = g[1];
    dst[24] = g[2];
  }
}

// ---------------------------------------------------------------------------
// Tensor-core element contraction.
// Operand tiles: row c of a tile = basis column c of the element, K = the
// chunk's quadrature points; 10 tiles per stage:
//   0/1 Y0 hi/lo, 2/3 Y1, 4/5 Y2 (Y_d = sqrt(w/2) dphi/dx_d), 6/7 Z (sqrt(w) phi),
//   8/9 ZV (V sqrt(w) phi).
// Per 8-point K-step and M-tile:  H += ZV^T Z (all columns),
//   H[:, 64:] += sum_d Y_d^T Y_d[64:],  S[:, 64:] += Z^T Z[64:].
// Inputs of each chunk (the FP32 Psi table block and the point data) are
// brought into shared memory one chunk ahead by the TMA engine (1D bulk
// copies completing on an mbarrier), so the fill reads shared memory only.
// ---------------------------------------------------------------------------
struct TcShared {
  uint64_t sbar[NSTAGE];  // operand stage free (MMA commit)
  uint64_t ibar[NSTAGE];  // chunk inputs arrived (bulk copy)
  uint32_t tmem;
  int pad;
  float L[16][3][4];   // per chunk point: 1D Lagrange values
  float dL[16][3][4];  // and slopes (times 2/h)
  float xi[16][3];
  float sw2[16], sw[16], v[16];
};

template <int R>
__global__ void __launch_bounds__(TC_NT, 1) k_assemble_tc(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ ecol,
    const int32_t *__restrict__ aoff, const int64_t *__restrict__ toff32,
    const float *__restrict__ psi, const int64_t *__restrict__ soff,
    const int32_t *__restrict__ smap, const double *__restrict__ V, float sx, float sy, float sz,
    int nelem_list, int in_bytes, int want, double *__restrict__ H, double *__restrict__ S,
    unsigned *err) {
  constexpr int KC = 2048 / R;             // chunk of quadrature points (16 or 8)
  constexpr int TILE = R * KC * 4;         // bytes per tile
  constexpr uint32_t LBO = 128;            // next core matrix along K
  constexpr uint32_t SBO = (KC / 4) * 128; // next 8-row group along M/N
  // Tensor-core FP32 accumulation does not round to nearest; its error grows
  // with the number of MMAs summed into one accumulator.  With the 128-row
  // tile the large hi*hi products and the small cross products go to
  // separate accumulators (cross terms are ~2^-11 smaller, so their error is
  // negligible) and the two are added in FP64 by the epilogue.
  constexpr bool SPLIT = (R == 128);
  constexpr uint32_t TCOLS = 512;
  constexpr uint32_t HX_COL = SPLIT ? 128 : 0;    // cross-term H accumulator
  constexpr uint32_t S_COL = 256;                 // hi*hi S accumulator
  constexpr uint32_t SX_COL = SPLIT ? 320 : 256;  // cross-term S accumulator
  static_assert(NTILES * TILE == STAGE_BYTES, "stage size");

  extern __shared__ __align__(16) unsigned char dsm[];
  unsigned char *stages = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  unsigned char *inbuf = stages + NSTAGE * STAGE_BYTES;   // NSTAGE x in_bytes
  TcShared &sh = *reinterpret_cast<TcShared *>(inbuf + NSTAGE * in_bytes);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (blockIdx.x >= (unsigned)nelem_list) return;
  const int e = order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int Qp = (int)(qpoff[e + 1] - qpoff[e]);
  const int A = aoff[e + 1] - aoff[e];
  const int n = (int)(doff[e + 1] - doff[e]);
  const int nenr = n - 64;
  const int npad = (n + 15) & ~15;
  const int nenr16 = (nenr + 15) & ~15;
  if (n > R || A * 4 * KC * 4 + KC * 16 > in_bytes) {
    if (tid == 0) set_err(err, DEVERR_SHAPE);
    return;
  }
  const int32_t *ec = ecol + (doff[e] - 64ll * e);
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  const float s3[3] = {sx, sy, sz};
  const int psi_off = A * 4 * KC * 4;  // bytes of the Psi block inside an input buffer

  // zero the input buffers once (stale but finite data is harmless later)
  for (int i = tid; i < NSTAGE * in_bytes / 16; i += TC_NT)
    reinterpret_cast<float4 *>(inbuf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) tmem_alloc(&sh.tmem, TCOLS);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&sh.sbar[s], 1);
      mbar_init(&sh.ibar[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tH = sh.tmem;
  const uint32_t tHx = sh.tmem + HX_COL;
  const uint32_t tS = sh.tmem + S_COL;
  const uint32_t tSx = sh.tmem + SX_COL;
  const uint32_t sbase = smem_u32(stages);
  const uint32_t idH = idesc_tf32(128, npad);
  const uint32_t idE = idesc_tf32(128, nenr16 > 0 ? nenr16 : 16);

  const int nch = (Qp + KC - 1) / KC;       // chunks per pass
  const int nmt = (n + 127) / 128;          // M-tile passes
  const int NJ = nch * nmt;
  // thread 0: bulk-load the inputs of flat chunk j into buffer j % 2
  auto issue_load = [&](int j) {
    const int qc = (j % nch) * KC;
    const int npt = min(KC, Qp - qc);        // a multiple of 8
    unsigned char *dst = inbuf + (j & 1) * in_bytes;
    const uint32_t pbytes = (uint32_t)(A * 4 * npt * 4);
    const uint32_t qbytes = (uint32_t)(npt * 16);
    mbar_expect_tx(&sh.ibar[j & 1], pbytes + qbytes);
    if (pbytes) bulk_g2s(dst, pe + (int64_t)(qc >> 3) * A * 32, pbytes, &sh.ibar[j & 1]);
    bulk_g2s(dst + psi_off, qe + qc, qbytes, &sh.ibar[j & 1]);
  };
  if (tid == 0) issue_load(0);

  bool ok = true;
  for (int j = 0; j < NJ && ok; ++j) {
    const int stg = j & 1;
    const int mt = j / nch;
    const int qc = (j % nch) * KC;
    unsigned char *sp = stages + stg * STAGE_BYTES;
    const float *ip = reinterpret_cast<const float *>(inbuf + stg * in_bytes);
    const float4 *iq = reinterpret_cast<const float4 *>(inbuf + stg * in_bytes + psi_off);
    // V of this chunk (plain loads, consumed after the barrier below)
    float vload = 0.0f;
    if (tid >= 64 && tid < 64 + KC) {
      const int q = qc + tid - 64;
      if (V && q < Q) vload = (float)V[q0 + q];
    }
    int good = 1;
    if (tid == 0) {
      // operand stage free: MMAs of chunk j-2 done; inputs of chunk j here
      if (j >= 2 && !mbar_wait(&sh.sbar[stg], ((j >> 1) - 1) & 1)) good = 0;
      if (good && !mbar_wait(&sh.ibar[stg], (j >> 1) & 1)) good = 0;
      if (good && j + 1 < NJ) issue_load(j + 1);
    }
    if (!__syncthreads_and(good)) {
      ok = false;
      break;
    }
    // per-point tables of the chunk
    if (tid < KC * 3) {
      const int qq = tid / 3, d = tid - 3 * qq;
      const float4 xq = iq[qq];
      const float xv = d == 0 ? xq.x : (d == 1 ? xq.y : xq.z);
      float L[4], dL[4];
      lagrange3f(xv, L, dL);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sh.L[qq][d][c] = L[c];
        sh.dL[qq][d][c] = dL[c] * s3[d];
      }
      sh.xi[qq][d] = xv;
    } else if (tid >= 64 && tid < 64 + KC) {
      const int qq = tid - 64;
      const float ww = (qc + qq < Qp) ? iq[qq].w : 0.0f;
      sh.sw2[qq] = sqrtf(0.5f * ww);
      sh.sw[qq] = sqrtf(ww);
      sh.v[qq] = vload;
    }
    __syncthreads();
    // fill rows < npad: each warp writes whole core matrices (8 rows x 4
    // points): lane -> (row c%8 = lane/4, point q%4 = lane%4), conflict-free
    const int ncm = (npad / 8) * (KC / 4);
    for (int cm = warp; cm < ncm; cm += TC_NT / 32) {
      const int rg = cm / (KC / 4), kg = cm - rg * (KC / 4);
      const int c = rg * 8 + (lane >> 2);
      const int qq = kg * 4 + (lane & 3);
      float b = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
      if (c < 64) {
        const int ia = c & 3, ib = (c >> 2) & 3, ic = c >> 4;
        const float lx = sh.L[qq][0][ia], ly = sh.L[qq][1][ib], lz = sh.L[qq][2][ic];
        b = lx * ly * lz;
        gx = sh.dL[qq][0][ia] * ly * lz;
        gy = lx * sh.dL[qq][1][ib] * lz;
        gz = lx * ly * sh.dL[qq][2][ic];
      } else if (c < n) {
        const int code = ec[c - 64];
        const int slot = code >> 3, lv = code & 7;
        const float *pp = ip + (((qq >> 3) * A + slot) * 4) * 8 + (qq & 7);
        const float p0 = pp[0], p1 = pp[8], p2 = pp[16], p3 = pp[24];
        float hh[3], dh[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int bit = (lv >> d) & 1;
          const float xv = sh.xi[qq][d];
          hh[d] = bit ? 0.5f * (1.0f + xv) : 0.5f * (1.0f - xv);
          dh[d] = (bit ? 0.5f : -0.5f) * s3[d];
        }
        const float phi = hh[0] * hh[1] * hh[2];
        b = phi * p0;
        gx = dh[0] * hh[1] * hh[2] * p0 + phi * p1;
        gy = hh[0] * dh[1] * hh[2] * p0 + phi * p2;
        gz = hh[0] * hh[1] * dh[2] * p0 + phi * p3;
      }
      const float r2 = sh.sw2[qq], r1 = sh.sw[qq];
      const float val[5] = {r2 * gx, r2 * gy, r2 * gz, r1 * b, sh.v[qq] * (r1 * b)};
      const uint32_t off = (uint32_t)rg * SBO + (uint32_t)kg * LBO + (uint32_t)lane * 4;
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        const float hi = tf32_rn(val[t]);
        const float lo = tf32_rn(val[t] - hi);
        *reinterpret_cast<float *>(sp + (2 * t) * TILE + off) = hi;
        *reinterpret_cast<float *>(sp + (2 * t + 1) * TILE + off) = lo;
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t st = sbase + stg * STAGE_BYTES;
      const uint32_t moff = (uint32_t)mt * 16u * SBO;   // M-tile: 128 rows
      const uint32_t eoff = 8u * SBO;                   // enrichment rows start at 64
#pragma unroll
      for (int ks = 0; ks < KC / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 2u * LBO;
        const uint32_t first = (qc == 0 && ks == 0) ? 0u : 1u;
        auto D = [&](int t, uint32_t extra) { return sdesc(st + t * TILE + ko + extra, LBO, SBO); };
        // H_V = ZV^T Z over all columns (hi*hi, then hi*lo + lo*hi)
        const uint32_t fx = SPLIT ? first : 1u;
        mma_tf32(tH, D(8, moff), D(6, 0), idH, first);
        mma_tf32(tHx, D(8, moff), D(7, 0), idH, fx);
        mma_tf32(tHx, D(9, moff), D(6, 0), idH, 1u);
        if (nenr > 0) {
          // T on the enrichment columns: sum_d Y_d^T Y_d[64:]
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            mma_tf32(tH + 64, D(2 * d, moff), D(2 * d, eoff), idE, 1u);
            mma_tf32(tHx + 64, D(2 * d, moff), D(2 * d + 1, eoff), idE, 1u);
            mma_tf32(tHx + 64, D(2 * d + 1, moff), D(2 * d, eoff), idE, 1u);
          }
          // S on the enrichment columns: Z^T Z[64:]
          mma_tf32(tS, D(6, moff), D(6, eoff), idE, first);
          mma_tf32(tSx, D(6, moff), D(7, eoff), idE, SPLIT ? first : 1u);
          mma_tf32(tSx, D(7, moff), D(6, eoff), idE, 1u);
        }
      }
      mma_commit(&sh.sbar[stg]);
    }
    if (j % nch != nch - 1) continue;
    // ---- end of an M-tile pass: drain the accumulators ----
    {
      int good2 = 1;
      if (tid == 0) good2 = mbar_wait(&sh.sbar[stg], (j >> 1) & 1) ? 1 : 0;
      if (!__syncthreads_and(good2)) {
        ok = false;
        break;
      }
    }
    tc_fence_after();
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (rows), column blocks
    // of 16 alternate between warps w and w+4
    const int quarter = warp & 3, half = warp >> 2;
    const int r = mt * 128 + quarter * 32 + lane;
    const uint32_t lanebase = (uint32_t)(quarter * 32) << 16;
    const int32_t *m = smap + soff[e];
    for (int cb = half; cb * 16 < npad; cb += 2) {
      float hv[16], sv[16], hx[16], sx2[16];
      tmem_ld16(tH + lanebase + cb * 16, hv);
      if (SPLIT) tmem_ld16(tHx + lanebase + cb * 16, hx);
      const bool enr_blk = cb * 16 >= 64;
      if (enr_blk && nenr > 0) {
        tmem_ld16(tS + lanebase + (cb * 16 - 64), sv);
        if (SPLIT) tmem_ld16(tSx + lanebase + (cb * 16 - 64), sx2);
      }
      if (r < n) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = cb * 16 + i;
          if (c >= n) break;
          const bool own = (c < 64) ? (c <= r && r < 64) : (r < 64 || c <= r);
          if (!own) continue;
          const int32_t sij = m[(int64_t)r * n + c];
          const int32_t sji = m[(int64_t)c * n + r];
          if (want & PUFE_WANT_H) {
            const double hval = SPLIT ? (double)hv[i] + (double)hx[i] : (double)hv[i];
            atomicAdd(H + sij, hval);
            if (c != r) atomicAdd(H + sji, hval);
          }
          if (enr_blk && (want & PUFE_WANT_S)) {
            const double sval = SPLIT ? (double)sv[i] + (double)sx2[i] : (double)sv[i];
            atomicAdd(S + sij, sval);
            if (c != r) atomicAdd(S + sji, sval);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (!ok && tid == 0) {
    set_err(err, DEVERR_TIMEOUT);
    // give copies and MMAs still in flight one more bounded wait
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_wait(&sh.sbar[s], 0);
      mbar_wait(&sh.ibar[s], 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(sh.tmem, TCOLS);
  }
}

// ---------------------------------------------------------------------------
// K4' (FP32): density, one CTA per element, one thread per point.
// ---------------------------------------------------------------------------
constexpr int DEN_NT = 128;

__global__ void __launch_bounds__(DEN_NT) k_density_f32(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ dofs,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const double *__restrict__ C, int64_t ldc, const double *__restrict__ f, int nocc, int noccp,
    double *__restrict__ rho) {
  extern __shared__ __align__(16) float fsm[];
  const int e = order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int A = aoff[e + 1] - aoff[e];
  const int n = (int)(doff[e + 1] - doff[e]);
  const int nenr = n - 64;
  const int32_t *ec = ecol + (doff[e] - 64ll * e);
  const int32_t *dl = dofs + doff[e];
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  float *Cs = fsm;              // n x noccp
  float *fs = Cs + n * noccp;   // noccp
  for (int k = threadIdx.x; k < n * noccp; k += DEN_NT) {
    const int j = k / noccp, kk = k - j * noccp;
    Cs[k] = (kk < nocc) ? (float)C[(int64_t)dl[j] * ldc + kk] : 0.0f;
  }
  for (int k = threadIdx.x; k < noccp; k += DEN_NT) fs[k] = (k < nocc) ? (float)f[k] : 0.0f;
  __syncthreads();
  for (int q = threadIdx.x; q < Q; q += DEN_NT) {
    const float4 x4 = qe[q];
    const float xq[3] = {x4.x, x4.y, x4.z};
    float L[3][4], dL[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) lagrange3f(xq[d], L[d], dL[d]);
    float pu[8];
#pragma unroll
    for (int lv = 0; lv < 8; ++lv) {
      float p = 1.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) p *= ((lv >> d) & 1) ? 0.5f * (1.0f + xq[d]) : 0.5f * (1.0f - xq[d]);
      pu[lv] = p;
    }
    const float *pq = pe + (int64_t)(q >> 3) * A * 32 + (q & 7);
    float r = 0.0f;
    for (int k0 = 0; k0 < noccp; k0 += 8) {
      float acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
#pragma unroll
      for (int c3 = 0; c3 < 4; ++c3)
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
          const float lyz = L[1][c2] * L[2][c3];
#pragma unroll
          for (int c1 = 0; c1 < 4; ++c1) {
            const float b = L[0][c1] * lyz;
            const float *cr = Cs + (c1 + 4 * c2 + 16 * c3) * noccp + k0;
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = fmaf(b, cr[k], acc[k]);
          }
        }
      for (int j = 0; j < nenr; ++j) {
        const int code = ec[j];
        const float b = pu[code & 7] * pq[(code >> 3) * 32];
        const float *cr = Cs + (64 + j) * noccp + k0;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fmaf(b, cr[k], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) r = fmaf(fs[k0 + k] * acc[k], acc[k], r);
    }
    rho[q0 + q] = (double)r;
  }
}

// ---------------------------------------------------------------------------
// K5' (FP32): Vbar_q = w_q b_q^T Hbar_e b_q.  One CTA per element: Hbar_e
// (gathered through the scatter map) and a chunk of 32 basis rows sit in
// shared memory; each thread owns a 4-point x 4-row register tile of
// t_qi = sum_j Hbar_ij b_qj and reduces b_qi t_qi into the point's sum.
// ---------------------------------------------------------------------------
constexpr int ADJ_NT = 256;
constexpr int ADJ_QB = 32;

__global__ void __launch_bounds__(ADJ_NT) k_adjoint_f32(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const double *__restrict__ w, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap,
    const double *__restrict__ Hbar, double *__restrict__ Vbar) {
  extern __shared__ __align__(16) float fsm[];
  const int e = order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int A = aoff[e + 1] - aoff[e];
  const int n = (int)(doff[e + 1] - doff[e]);
  const int n4 = (n + 3) & ~3;
  const int ldb = n4 + ((4 - (n4 & 31)) & 31);   // row stride = 4 mod 32 banks
  const int32_t *ec = ecol + (doff[e] - 64ll * e);
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  const int32_t *m = smap + soff[e];
  float *Hs = fsm;                 // n4 x n4, zero padded
  float *Bq = Hs + n4 * n4;        // ADJ_QB x ldb
  float *acc = Bq + ADJ_QB * ldb;  // ADJ_QB
  for (int k = threadIdx.x; k < n4 * n4; k += ADJ_NT) {
    const int i = k / n4, j = k - i * n4;
    Hs[k] = (i < n && j < n) ? (float)Hbar[m[i * n + j]] : 0.0f;
  }
  const int nI = n4 / 4;
  const int ntile = (ADJ_QB / 4) * nI;
  for (int qc = 0; qc < Q; qc += ADJ_QB) {
    __syncthreads();
    for (int k = threadIdx.x; k < ADJ_QB * n4; k += ADJ_NT) {
      const int qq = k / n4, c = k - qq * n4;
      const int q = qc + qq;
      float b = 0.0f;
      if (q < Q && c < n) {
        const float4 x4 = qe[q];
        if (c < 64) {
          float L[4], dL[4], v = 1.0f;
          lagrange3f(x4.x, L, dL);
          v *= L[c & 3];
          lagrange3f(x4.y, L, dL);
          v *= L[(c >> 2) & 3];
          lagrange3f(x4.z, L, dL);
          b = v * L[c >> 4];
        } else {
          const int code = ec[c - 64];
          const int lv = code & 7;
          const float phi = (((lv & 1) ? 1.0f + x4.x : 1.0f - x4.x) *
                             ((lv & 2) ? 1.0f + x4.y : 1.0f - x4.y) *
                             ((lv & 4) ? 1.0f + x4.z : 1.0f - x4.z)) * 0.125f;
          b = phi * pe[((int64_t)(q >> 3) * A + (code >> 3)) * 32 + (q & 7)];
        }
      }
      Bq[qq * ldb + c] = b;
    }
    if (threadIdx.x < ADJ_QB) acc[threadIdx.x] = 0.0f;
    __syncthreads();
    for (int t = threadIdx.x; t < ntile; t += ADJ_NT) {
      const int tq = t & (ADJ_QB / 4 - 1), ti = t / (ADJ_QB / 4);
      const float *b0 = Bq + (4 * tq) * ldb;
      const float *h0 = Hs + (4 * ti) * n4;
      float a[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) a[x][y] = 0.0f;
      for (int j = 0; j < n4; j += 4) {
        float4 bv[4], hv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) bv[x] = *reinterpret_cast<const float4 *>(b0 + x * ldb + j);
#pragma unroll
        for (int y = 0; y < 4; ++y) hv[y] = *reinterpret_cast<const float4 *>(h0 + y * n4 + j);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y)
            a[x][y] += bv[x].x * hv[y].x + bv[x].y * hv[y].y + bv[x].z * hv[y].z + bv[x].w * hv[y].w;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float s = 0.0f;
#pragma unroll
        for (int y = 0; y < 4; ++y) s = fmaf(b0[x * ldb + 4 * ti + y], a[x][y], s);
        atomicAdd(acc + 4 * tq + x, s);
      }
    }
    __syncthreads();
    if (threadIdx.x < ADJ_QB && qc + (int)threadIdx.x < Q)
      Vbar[q0 + qc + threadIdx.x] = w[q0 + qc + threadIdx.x] * (double)acc[threadIdx.x];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
pufe_status launch_tabulate_f32(pufe_ctx *ctx, cudaStream_t st) {
  if (ctx->psi32_len == 0) return PUFE_OK;
  auto &D = ctx->d;
  k_tabulate_f32<<<(unsigned)ctx->nelem, 256, 0, st>>>(
      D.qpoff, D.qdat, D.aoff, D.alist, D.toff32, D.orbf, D.eorig, (float)ctx->a[0],
      (float)ctx->a[1], (float)ctx->a[2], (float)ctx->h[0], (float)ctx->h[1], (float)ctx->h[2],
      D.psi32);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_assemble_tc(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                               cudaStream_t st) {
  auto &D = ctx->d;
  if (!ctx->fe_exact)
    return fail(PUFE_EINVAL,
                "PUFE_TF32X3 needs every (sub)cell rule to have >= 4 points per axis");
  if (ctx->max_basis > 256) return fail(PUFE_EINVAL, "PUFE_TF32X3 supports n_e <= 256");
  // constant FE-FE blocks: start from the precomputed global T0 / S0
  const size_t bytes = (size_t)ctx->nnz * sizeof(double);
  if (what & PUFE_WANT_H) PUFE_CUDA_TRY(cudaMemcpyAsync(H, D.T0, bytes, cudaMemcpyDeviceToDevice, st));
  if (what & PUFE_WANT_S) PUFE_CUDA_TRY(cudaMemcpyAsync(S, D.S0, bytes, cudaMemcpyDeviceToDevice, st));
  const float sx = (float)(2.0 / ctx->h[0]), sy = (float)(2.0 / ctx->h[1]),
              sz = (float)(2.0 / ctx->h[2]);
  auto smem_for = [&](int KC, int &in_bytes) {
    in_bytes = ((ctx->max_alpha * 4 * KC * 4 + KC * 16) + 127) & ~127;
    return (size_t)1024 + NSTAGE * STAGE_BYTES + NSTAGE * in_bytes + sizeof(TcShared);
  };
  // elements are ordered with n_e > 128 first (256-row tile), then the rest
  const int nbig = ctx->n_big;
  if (nbig > 0) {
    int inb = 0;
    const size_t sm = smem_for(8, inb);
    if (sm > 227 * 1024) return fail(PUFE_EINVAL, "too many enrichments per element for TF32X3");
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_assemble_tc<256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_assemble_tc<256><<<nbig, TC_NT, sm, st>>>(D.order, D.qoff, D.qpoff, D.qdat, D.doff, D.ecol,
                                                D.aoff, D.toff32, D.psi32, D.soff, D.smap, V, sx,
                                                sy, sz, nbig, inb, what, H, S, D.err);
    PUFE_CUDA_TRY(cudaGetLastError());
  }
  const int nsmall = (int)ctx->nelem - nbig;
  if (nsmall > 0) {
    int inb = 0;
    const size_t sm = smem_for(16, inb);
    if (sm > 227 * 1024) return fail(PUFE_EINVAL, "too many enrichments per element for TF32X3");
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_assemble_tc<128>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_assemble_tc<128><<<nsmall, TC_NT, sm, st>>>(D.order + nbig, D.qoff, D.qpoff, D.qdat,
                                                  D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
                                                  D.soff, D.smap, V, sx, sy, sz, nsmall, inb,
                                                  what, H, S, D.err);
    PUFE_CUDA_TRY(cudaGetLastError());
  }
  return PUFE_OK;
}

pufe_status launch_density_tc(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f,
                              int nocc, double *rho, cudaStream_t st) {
  auto &D = ctx->d;
  const int noccp = (nocc + 7) & ~7;
  const size_t sm = ((size_t)ctx->max_basis * noccp + noccp) * sizeof(float);
  PUFE_CUDA_TRY(
      cudaFuncSetAttribute(k_density_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_density_f32<<<(unsigned)ctx->nelem, DEN_NT, sm, st>>>(D.order, D.qoff, D.qpoff, D.qdat,
                                                          D.doff, D.dofs, D.ecol, D.aoff,
                                                          D.toff32, D.psi32, C, ldc, f, nocc,
                                                          noccp, rho);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_adjoint_tc(pufe_ctx *ctx, const double *Hbar, double *Vbar, cudaStream_t st) {
  auto &D = ctx->d;
  const int n4 = (ctx->max_basis + 3) & ~3;
  const int ldb = n4 + 36;
  const size_t sm = ((size_t)n4 * n4 + (size_t)ADJ_QB * ldb + ADJ_QB) * sizeof(float);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "n_e too large for the FP32 adjoint kernel");
  PUFE_CUDA_TRY(
      cudaFuncSetAttribute(k_adjoint_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_adjoint_f32<<<(unsigned)ctx->nelem, ADJ_NT, sm, st>>>(D.order, D.qoff, D.qpoff, D.qdat, D.w,
                                                          D.doff, D.ecol, D.aoff, D.toff32,
                                                          D.psi32, D.soff, D.smap, Hbar, Vbar);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

}  // namespace pufe
