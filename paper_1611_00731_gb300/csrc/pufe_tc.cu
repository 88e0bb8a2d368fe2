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

#include <algorithm>
#include <mutex>

#include "pufe_internal.h"

namespace pufe {

namespace {

constexpr int NTILES = 10;          // Y0,Y1,Y2,Z,ZV x (hi, lo)
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

// Wait for completion `parity` of an mbarrier, giving up after `limit` ns.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t *bar, uint32_t parity, uint64_t limit) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (globaltimer() - t0 > limit) return false;
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  return mbar_wait_ns(bar, parity, WAIT_NS);
}

// Diagnostics of the timeout path: one thread waits, with the bounded wait
// of the pipelined kernels, on an mbarrier that expects one arrival that
// never comes; when the wait gives up it sets DEVERR_TIMEOUT, completes the
// phase itself (so nothing is left pending) and returns.
__global__ void k_wait_probe(uint64_t limit, unsigned *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait_ns(&bar, 0, limit)) {
    atomicOr(err, DEVERR_TIMEOUT);
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(
                     smem_u32(&bar))
                 : "memory");
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
constexpr int TAB_NT = 256;
// slots one CTA's chunk can touch: padded elements hold a multiple of 8
// points, so a chunk of TAB_CHUNK items spans at most TAB_CHUNK / 8 + 2 slots
constexpr int TAB_SLOTS = TAB_CHUNK / 8 + 2;

// 40 registers (six CTAs per SM): measured 39.6 -> 33.4 us on the 12^3
// rocksalt cell against the unbounded 80-register form; a 32-register cap
// spills and is slower (56 us)
__global__ void __launch_bounds__(TAB_NT, 6) k_tabulate_f32(
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const int32_t *__restrict__ aoff, const int32_t *__restrict__ alist,
    const int64_t *__restrict__ toff32, const OrbitalF *__restrict__ orbf,
    const float *__restrict__ eorig, float ax, float ay, float az, float hx, float hy, float hz,
    const int32_t *__restrict__ tblk, int nelem, float *__restrict__ psi) {
  const float av[3] = {ax, ay, az};
  const float inv_a[3] = {1.0f / ax, 1.0f / ay, 1.0f / az};
  const float hh[3] = {0.5f * hx, 0.5f * hy, 0.5f * hz};
  // CTA b takes the (slot, padded point) items [c TAB_CHUNK, (c + 1) TAB_CHUNK)
  // of element e, c = b - tblk[e] (tblk: CTAs per element, prefix summed), so
  // elements with many points and slots spread over many CTAs.  The orbital
  // and the element-origin displacement of each slot the chunk touches are
  // staged in shared memory once per CTA.
  __shared__ int s_e;
  __shared__ OrbitalF s_orb[TAB_SLOTS];
  __shared__ float s_eo[TAB_SLOTS][6];
  if (threadIdx.x == 0) {
    int lo_e = 0, hi_e = nelem;   // tblk[lo_e] <= b < tblk[hi_e]
    while (hi_e - lo_e > 1) {
      const int mid = (lo_e + hi_e) >> 1;
      if (tblk[mid] <= (int)blockIdx.x) lo_e = mid; else hi_e = mid;
    }
    s_e = lo_e;
  }
  __syncthreads();
  const int e = s_e;
  const int64_t q0 = qpoff[e];
  const int Qp = (int)(qpoff[e + 1] - q0);
  const int a0 = aoff[e];
  const int A = aoff[e + 1] - a0;
  float *out = psi + 4 * toff32[e];
  const int base = ((int)blockIdx.x - tblk[e]) * TAB_CHUNK;
  const int end = min(base + TAB_CHUNK, Qp * A);
  if (base >= end) return;   // uniform over the CTA
  const int sl0 = base / Qp;
  const int nsl = (end - 1) / Qp - sl0 + 1;
  // the stage holds every slot of a chunk unless an element's padded point
  // count is below 8, which the layout excludes; such a chunk reads the
  // orbital data from global memory instead
  const bool staged = nsl <= TAB_SLOTS;
  if (staged) {
    for (int t = threadIdx.x; t < nsl * 7; t += TAB_NT) {
      const int s = t / 7, c = t - 7 * s;
      if (c == 6)
        s_orb[s] = orbf[alist[a0 + sl0 + s]];
      else
        s_eo[s][c] = eorig[8 * (int64_t)(a0 + sl0 + s) + c];
    }
  }
  __syncthreads();
  int idx = base + threadIdx.x;
  int slot = idx / Qp, q = idx - slot * Qp;
  for (; idx < end; idx += TAB_NT) {
    OrbitalF o;
    float eo[6];
    if (staged) {
      o = s_orb[slot - sl0];
#pragma unroll
      for (int c = 0; c < 6; ++c) eo[c] = s_eo[slot - sl0][c];
    } else {
      o = orbf[alist[a0 + slot]];
#pragma unroll
      for (int c = 0; c < 6; ++c) eo[c] = eorig[8 * (int64_t)(a0 + slot) + c];
    }
    const float4 xq = qdat[q0 + q];
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
    // the next item of this thread, TAB_NT items on
    q += TAB_NT;
    while (q >= Qp) {
      q -= Qp;
      ++slot;
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core element contraction for elements with n_e > 128 (up to 256
// basis functions): persistent, warp-specialized.
//
// The FE-FE blocks are done elsewhere (exact kinetic constants and the
// sum-factorized V term); this kernel computes the enrichment strip:
//   H[:, 64:] = ZV^T Z[64:] + sum_d Y_d^T Y_d[64:],   S[:, 64:] = Z^T Z[64:],
// with, per 8-point chunk, Y_d = sqrt(w/2) dphi/dx_d, Z = sqrt(w) phi and
// ZV = V Z for every basis column (rows of the A operand, two 128-row
// M-tiles) and the enrichment columns only (rows of the B operand), each
// split into two TF32 terms (three MMAs per product: hi*hi, hi*lo, lo*hi).
//
// Roles (one CTA per SM, elements taken round-robin from the work list):
//   warps 0-7   fill: per chunk, wait for the chunk's inputs (in shared
//               memory, brought by the loader) and a free operand stage,
//               write the operand core matrices into shared memory, then
//               signal "stage full" and "input free";
//   warp 8      MMA: one lane issues tcgen05.mma per full stage, commits to
//               "stage empty" and, at the end of an M-tile, "acc full";
//   warps 9-12  epilogue: drain the accumulators, add them into the FP64 CSR
//               values, signal "acc empty";
//   warp 13     loader: 1D TMA bulk copies of each chunk's inputs (Psi table
//               block, per-point table, V) into a ring of input buffers.
// All waits are bounded (2 s); a timeout sets the device error flag and every
// role leaves its loop.
// ---------------------------------------------------------------------------
constexpr int WS_MMA_WARP = 8;
constexpr int WS_EPI_WARP0 = 9;       // warps 9-12
constexpr int WS_LOAD_WARP = 13;
constexpr int WS_NT = 14 * 32;
constexpr int WS_KC = 8;              // quadrature points per chunk (one K-step)
constexpr int WS_NIN = 6;             // input buffers

struct WsShared {
  uint64_t sfull[4], sempty[4], ibar[WS_NIN], ifree[WS_NIN], afull, aempty;
  uint32_t tmem;
  int abort;      // any role gave up: everyone leaves
};
// after WsShared: the epilogue warps' transpose buffers (4 x 32 x 17 float2)

// FP32 copy of V on the padded point layout (zeros on padding points) for the
// elements order[0 .. gridDim.x), so that the tensor-core kernel's bulk
// copies can bring it in with the other inputs.
__global__ void k_pack_v(const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
                         const int64_t *__restrict__ qpoff, const double *__restrict__ V,
                         float *__restrict__ vpad) {
  const int64_t e = order[blockIdx.x];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int Qp = (int)(qpoff[e + 1] - qpoff[e]);
  for (int q = threadIdx.x; q < Qp; q += blockDim.x)
    vpad[qpoff[e] + q] = (q < Q && V) ? (float)V[q0 + q] : 0.0f;
}

struct ElemInfo {
  int e, Q, Qp, A, n, nenr, npad, nenr16, nch, nmt, c0;
  int64_t q0;
  bool ok;   // the kernel can take this element
  bool go;   // ok and it has enrichment columns (FE-only elements need no strip)
};

// work item k: chunks [c0, c1) of element order[items[3k]] (chunks of WS_KC
// padded points)
__device__ __forceinline__ ElemInfo elem_info(const int32_t *order, const int32_t *items, int k,
                                              const int64_t *qoff, const int64_t *qpoff,
                                              const int32_t *aoff, const int64_t *doff, int amax) {
  ElemInfo I;
  I.e = order[items[3 * k]];
  I.q0 = qoff[I.e];
  I.Q = (int)(qoff[I.e + 1] - I.q0);
  I.Qp = (int)(qpoff[I.e + 1] - qpoff[I.e]);
  I.A = aoff[I.e + 1] - aoff[I.e];
  I.n = (int)(doff[I.e + 1] - doff[I.e]);
  I.nenr = I.n - 64;
  I.npad = (I.n + 15) & ~15;
  I.nenr16 = (I.nenr + 15) & ~15;
  I.c0 = items[3 * k + 1];
  I.nch = items[3 * k + 2] - I.c0;
  I.nmt = (I.n + 127) / 128;
  I.ok = I.n <= 256 && I.A <= amax && I.nch > 0 && (I.c0 + I.nch) * WS_KC <= I.Qp;
  I.go = I.ok && I.nenr > 0;
  return I;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}



__global__ void __launch_bounds__(WS_NT, 1) k_assemble_tc(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float *__restrict__ ptab,
    const float *__restrict__ vpad, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap, float sx, float sy,
    float sz, const int32_t *__restrict__ items, int nelem_list, int amax, int in_bytes,
    int want, double *__restrict__ H, double *__restrict__ S, unsigned *err) {
  constexpr int R = 256;                      // basis rows of the tile (n_e <= 256)
  constexpr int KC = WS_KC;
  constexpr int TILE = R * KC * 4;            // bytes per SMEM tile
  constexpr int NBT = NTILES;                 // SMEM tiles per stage
  constexpr int STG = NBT * TILE;             // bytes per stage
  constexpr int NSTG = 2;                     // operand stages
  constexpr uint32_t LBO = 128;               // next core matrix along K
  constexpr uint32_t SBO = (KC / 4) * 128;    // next 8-row group along M/N
  constexpr uint32_t TCOLS = 512;
  constexpr uint32_t S_COL = 256;
  static_assert(NSTG * STG <= 163840, "stage memory");

  extern __shared__ __align__(16) unsigned char dsm[];
  unsigned char *stages = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  unsigned char *inbuf = stages + NSTG * STG;
  WsShared &sh = *reinterpret_cast<WsShared *>(inbuf + WS_NIN * in_bytes);
  float2(*epi)[32][17] = reinterpret_cast<float2(*)[32][17]>(reinterpret_cast<unsigned char *>(&sh) +
                                                            sizeof(WsShared));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float s3[3] = {sx, sy, sz};
  const int G = gridDim.x;

  // ---- set-up ---------------------------------------------------------------
  for (int i = tid; i < WS_NIN * in_bytes / 16; i += WS_NT)
    reinterpret_cast<float4 *>(inbuf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == WS_MMA_WARP) tmem_alloc(&sh.tmem, TCOLS);
  if (tid == 0) {
    for (int i = 0; i < NSTG; ++i) {
      mbar_init(&sh.sfull[i], 8);    // one arrival per fill warp
      mbar_init(&sh.sempty[i], 1);
    }
    for (int i = 0; i < WS_NIN; ++i) {
      mbar_init(&sh.ibar[i], 1);
      mbar_init(&sh.ifree[i], 8);    // one arrival per fill warp
    }
    mbar_init(&sh.afull, 1);
    mbar_init(&sh.aempty, 4);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp < 8) {
    // ======================= fill warps =======================
    // Each warp waits for the chunk's inputs and a free stage on its own and
    // signals completion with its own arrival, so warps never meet at a
    // CTA-wide barrier inside the loop and may drift apart by up to the
    // number of stages.
    int t = 0;
    bool run = true;
    for (int k = blockIdx.x; k < nelem_list && run; k += G) {
      const ElemInfo I = elem_info(order, items, k, qoff, qpoff, aoff, doff, amax);
      if (!I.ok) {
        if (tid == 0) set_err(err, DEVERR_SHAPE);
        continue;
      }
      if (!I.go) continue;
      const int32_t *ecs = ecol + (doff[I.e] - 64ll * I.e);
      for (int mt = 0; mt < I.nmt && run; ++mt) {
        for (int c = 0; c < I.nch; ++c, ++t) {
          const int s = t % NSTG, b = t % WS_NIN;
          unsigned char *sp = stages + s * STG;
          const float *ip = reinterpret_cast<const float *>(inbuf + b * in_bytes);
          const float *pt = ip + I.A * 4 * KC;   // per point: 32 floats
          const float *vq = pt + 32 * KC;        // per point: V
          int good = 1;
          if (lane == 0) {
            good = !*(volatile int *)&sh.abort;
            if (good) good = mbar_wait(&sh.ibar[b], (t / WS_NIN) & 1);
            if (good && t >= NSTG) good = mbar_wait(&sh.sempty[s], ((t / NSTG) - 1) & 1);
            if (!good) {
              set_err(err, DEVERR_TIMEOUT);
              atomicExch(&sh.abort, 1);
            }
          }
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            run = false;
            break;
          }
          tc_fence_after();
          // 256-row tile: every operand in shared memory, core matrices of
          // 8 rows x 4 points, lane -> (row = lane/4, point = lane%4)
          constexpr int CMW = R / 32;
          const int ncm = (I.npad / 8) * (KC / 4);
#pragma unroll
          for (int u = 0; u < CMW; ++u) {
            const int cm = warp + 8 * u;
            if (cm >= ncm) break;
            const int rg = cm >> 1, kg = cm & 1;
            const int cidx = rg * 8 + (lane >> 2);
            const int qq = kg * 4 + (lane & 3);
            const float *pq = pt + 32 * qq;
            float bv = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
            if (cidx < 64) {
              const int ia = cidx & 3, ib = (cidx >> 2) & 3, ic = cidx >> 4;
              const float lx = pq[ia], ly = pq[4 + ib], lz = pq[8 + ic];
              bv = lx * ly * lz;
              gx = pq[12 + ia] * ly * lz;
              gy = lx * pq[16 + ib] * lz;
              gz = lx * ly * pq[20 + ic];
            } else if (cidx < I.n) {
              const int code = ecs[cidx - 64];
              const int slot = code >> 3, lv = code & 7;
              const float *pp = ip + (slot * 4) * 8 + qq;
              const float p0 = pp[0], p1 = pp[8], p2 = pp[16], p3 = pp[24];
              float hh[3], dh[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                const int bit = (lv >> d) & 1;
                const float xv = pq[24 + d];
                hh[d] = bit ? 0.5f * (1.0f + xv) : 0.5f * (1.0f - xv);
                dh[d] = (bit ? 0.5f : -0.5f) * s3[d];
              }
              const float phi = hh[0] * hh[1] * hh[2];
              bv = phi * p0;
              gx = dh[0] * hh[1] * hh[2] * p0 + phi * p1;
              gy = hh[0] * dh[1] * hh[2] * p0 + phi * p2;
              gz = hh[0] * hh[1] * dh[2] * p0 + phi * p3;
            }
            const float r2 = pq[27], r1 = pq[28];
            const float val[5] = {r2 * gx, r2 * gy, r2 * gz, r1 * bv, vq[qq] * (r1 * bv)};
            const uint32_t off = (uint32_t)rg * SBO + (uint32_t)kg * LBO + (uint32_t)lane * 4;
#pragma unroll
            for (int tt = 0; tt < 5; ++tt) {
              const float hi = tf32_rn(val[tt]);
              *reinterpret_cast<float *>(sp + (2 * tt) * TILE + off) = hi;
              *reinterpret_cast<float *>(sp + (2 * tt + 1) * TILE + off) = tf32_rn(val[tt] - hi);
            }
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(&sh.sfull[s]);
            mbar_arrive(&sh.ifree[b]);
          }
        }
      }
    }
  } else if (warp == WS_MMA_WARP) {
    // ======================= MMA warp =======================
    if (lane == 0) {
      const uint32_t sbase = smem_u32(stages);
      int t = 0, a = 0;
      bool run = true;
      for (int k = blockIdx.x; k < nelem_list && run; k += G) {
        const ElemInfo I = elem_info(order, items, k, qoff, qpoff, aoff, doff, amax);
        if (!I.go) continue;
        const uint32_t idE = idesc_tf32(128, I.nenr16);
        const uint32_t tH = tmem, tS = tmem + S_COL;
        for (int mt = 0; mt < I.nmt && run; ++mt, ++a) {
          if (a > 0 && !mbar_wait(&sh.aempty, (a - 1) & 1)) {
            run = false;
            break;
          }
          tc_fence_after();
          for (int c = 0; c < I.nch; ++c, ++t) {
            const int s = t % NSTG;
            if (*(volatile int *)&sh.abort || !mbar_wait(&sh.sfull[s], (t / NSTG) & 1)) {
              run = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = sbase + s * STG;
            const uint32_t first = (c == 0) ? 0u : 1u;
            const uint32_t moff = (uint32_t)mt * 16u * SBO;   // M-tile: 128 rows
            const uint32_t eoff = 8u * SBO;                   // enrichment rows start at 64
            auto D = [&](int tt, uint32_t extra) { return sdesc(st + tt * TILE + extra, LBO, SBO); };
            mma_tf32(tH, D(8, moff), D(6, eoff), idE, first);
            mma_tf32(tH, D(8, moff), D(7, eoff), idE, 1u);
            mma_tf32(tH, D(9, moff), D(6, eoff), idE, 1u);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              mma_tf32(tH, D(2 * d, moff), D(2 * d, eoff), idE, 1u);
              mma_tf32(tH, D(2 * d, moff), D(2 * d + 1, eoff), idE, 1u);
              mma_tf32(tH, D(2 * d + 1, moff), D(2 * d, eoff), idE, 1u);
            }
            mma_tf32(tS, D(6, moff), D(6, eoff), idE, first);
            mma_tf32(tS, D(6, moff), D(7, eoff), idE, 1u);
            mma_tf32(tS, D(7, moff), D(6, eoff), idE, 1u);
            mma_commit(&sh.sempty[s]);
          }
          if (!run) break;
          mma_commit(&sh.afull);
        }
      }
      if (!run) {
        set_err(err, DEVERR_TIMEOUT);
        atomicExch(&sh.abort, 1);
      }
    }
    __syncwarp();
  } else if (warp < WS_LOAD_WARP) {
    // ======================= epilogue warps =======================
    const int quarter = warp & 3;
    const int ew = warp - WS_EPI_WARP0;
    const uint32_t lanebase = (uint32_t)(quarter * 32) << 16;
    float2(*stg)[17] = epi[ew];
    int a = 0;
    bool run = true;
    // Scatter one 32-row x 16-column block of the strip (columns cc = 64 +
    // 16 cb + i, all enrichment columns) into both CSR slots of every owned
    // pair: (r, cc) is owned when r < 64 (FE row) or cc <= r.  Two passes,
    // each keeping a warp's slots together: direct slots (r, cc): half-warp
    // h takes row 2 it + h, lanes run along 16 consecutive columns; mirror
    // slots (cc, r): lane = row, loop over the 16 columns.  All slot loads of
    // a pass are issued before its atomics.  For S only the FE rows are
    // scattered (fe_only): its E x E block comes from the FP64 kernel.
    auto owned = [&](int r, int cc, int n) { return r < n && cc < n && (r < 64 || cc <= r); };
    auto scatter_block = [&](const int32_t *m, int n, int rbase, int cb, double *out,
                             bool fe_only, auto value_of) {
      int sd[16];
#pragma unroll
      for (int it = 0; it < 16; ++it) {
        const int rl = 2 * it + (lane >> 4);
        const int r = rbase + rl, cc = 64 + cb * 16 + (lane & 15);
        sd[it] = (owned(r, cc, n) && (!fe_only || r < 64)) ? m[(int64_t)r * n + cc] : -1;
      }
#pragma unroll
      for (int it = 0; it < 16; ++it)
        if (sd[it] >= 0) atomicAdd(out + sd[it], value_of(2 * it + (lane >> 4), lane & 15));
      const int r = rbase + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int cc = 64 + cb * 16 + i;
        sd[i] = (cc != r && owned(r, cc, n) && (!fe_only || r < 64)) ? m[(int64_t)cc * n + r] : -1;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (sd[i] >= 0) atomicAdd(out + sd[i], value_of(lane, i));
    };
    for (int k = blockIdx.x; k < nelem_list && run; k += G) {
      const ElemInfo I = elem_info(order, items, k, qoff, qpoff, aoff, doff, amax);
      if (!I.go) continue;
      const int32_t *m = smap + soff[I.e];
      const int n = I.n;
      const int ncb = I.nenr16 / 16;
      for (int mt = 0; mt < I.nmt; ++mt, ++a) {
        int good = 1;
        if (lane == 0) good = (!*(volatile int *)&sh.abort && mbar_wait(&sh.afull, a & 1)) ? 1 : 0;
        good = __shfl_sync(0xffffffffu, good, 0);
        if (!good) {
          run = false;
          break;
        }
        tc_fence_after();
        const int rbase = mt * 128 + quarter * 32;
        for (int cb = 0; cb < ncb; ++cb) {
          for (int which = 0; which < 2; ++which) {
            if (which == 0 && !(want & PUFE_WANT_H)) continue;
            if (which == 1 && !(want & PUFE_WANT_S)) continue;
            float hv[16];
            tmem_ld16((which == 0 ? tmem : tmem + S_COL) + lanebase + cb * 16, hv);
#pragma unroll
            for (int i = 0; i < 16; ++i) stg[lane][i] = make_float2(hv[i], 0.0f);
            __syncwarp();
            scatter_block(m, n, rbase, cb, which == 0 ? H : S, which == 1, [&](int rl, int cl) {
              return (double)stg[rl][cl].x;
            });
            __syncwarp();
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.aempty);
      }
    }
  } else {
    // ======================= loader warp =======================
    if (lane == 0) {
      int lt = 0;
      bool run = true;
      for (int k = blockIdx.x; k < nelem_list && run; k += G) {
        const ElemInfo I = elem_info(order, items, k, qoff, qpoff, aoff, doff, amax);
        if (!I.go) continue;
        const float *lpsi = psi + 4 * toff32[I.e];
        const float *lpt = ptab + 32 * qpoff[I.e];
        const float *lv = vpad + qpoff[I.e];
        const uint32_t pbytes = (uint32_t)(I.A * 4 * KC * 4);
        for (int mt = 0; mt < I.nmt && run; ++mt) {
          for (int c = 0; c < I.nch; ++c, ++lt) {
            const int b = lt % WS_NIN;
            if (*(volatile int *)&sh.abort ||
                (lt >= WS_NIN && !mbar_wait(&sh.ifree[b], ((lt / WS_NIN) - 1) & 1))) {
              run = false;
              break;
            }
            const int qc = (I.c0 + c) * KC;
            unsigned char *dst = inbuf + b * in_bytes;
            mbar_expect_tx(&sh.ibar[b], pbytes + KC * 128 + KC * 4);
            if (pbytes) bulk_g2s(dst, lpsi + (int64_t)(qc >> 3) * I.A * 32, pbytes, &sh.ibar[b]);
            bulk_g2s(dst + pbytes, lpt + 32 * qc, KC * 128, &sh.ibar[b]);
            bulk_g2s(dst + pbytes + KC * 128, lv + qc, KC * 4, &sh.ibar[b]);
          }
        }
      }
      if (!run) {
        set_err(err, DEVERR_TIMEOUT);
        atomicExch(&sh.abort, 1);
      }
    }
    __syncwarp();
  }

  // ---- teardown -------------------------------------------------------------
  tc_fence_before();
  __syncthreads();
  if (warp == WS_MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

// shared-memory bytes of one k_assemble_tc launch
static size_t assemble_smem(int in_bytes) {
  const size_t stage = 2 * (size_t)(NTILES * 256 * WS_KC * 4);
  const size_t tail = (size_t)4 * 32 * 17 * 8;
  return (size_t)1024 + stage + WS_NIN * (size_t)in_bytes + sizeof(WsShared) + tail;
}

// ---------------------------------------------------------------------------
// K4' (FP32): density, one CTA per element, one thread per point.
// ---------------------------------------------------------------------------
constexpr int DEN_NT = 128;

// KC states k0 .. k0 + KC - 1 of one point added into r: sum_k f_k (sum_j b_j C_jk)^2 over
// the 64 tricubic columns (from the 1D factors L) and the enrichment columns
// (PU factor times the point's Psi value of the column's slot)
template <int KC>
__device__ __forceinline__ float density_states(const float (&L)[3][4], const float (&pu)[8],
                                                const float *pq, const int32_t *ec, int nenr,
                                                const float *Cb, const float *fs, int noccp,
                                                int k0, float r) {
  float acc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) acc[k] = 0.0f;
#pragma unroll
  for (int c3 = 0; c3 < 4; ++c3)
#pragma unroll
    for (int c2 = 0; c2 < 4; ++c2) {
      const float lyz = L[1][c2] * L[2][c3];
#pragma unroll
      for (int c1 = 0; c1 < 4; ++c1) {
        const float b = L[0][c1] * lyz;
        const float *cr = Cb + (c1 + 4 * c2 + 16 * c3) * noccp + k0;
#pragma unroll
        for (int k = 0; k < KC; ++k) acc[k] = fmaf(b, cr[k], acc[k]);
      }
    }
  for (int j = 0; j < nenr; ++j) {
    const int code = ec[j];
    const float b = pu[code & 7] * pq[(code >> 3) * 32];
    const float *cr = Cb + (64 + j) * noccp + k0;
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = fmaf(b, cr[k], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < KC; ++k) r = fmaf(fs[k0 + k] * acc[k], acc[k], r);
  return r;
}

template <bool BLOCH>
__global__ void __launch_bounds__(DEN_NT) k_density_f32(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const int64_t *__restrict__ doff, const int32_t *__restrict__ dofs,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const double *__restrict__ C, int64_t ldc, const double *__restrict__ f, int nocc, int noccp,
    double *__restrict__ rho, const int32_t *__restrict__ pitems, const double *__restrict__ Ci,
    const uint8_t *__restrict__ eshift, PhaseTab ph) {
  extern __shared__ __align__(16) float fsm[];
  // work item: points [qb, qend) of element order[k]
  const int e = order[pitems[3 * blockIdx.x]];
  const int qb = pitems[3 * blockIdx.x + 1];
  const int64_t q0 = qoff[e];
  const int Q = min((int)(qoff[e + 1] - q0), pitems[3 * blockIdx.x + 2]);
  const int A = aoff[e + 1] - aoff[e];
  const int n = (int)(doff[e + 1] - doff[e]);
  const int nenr = n - 64;
  const int32_t *ec = ecol + (doff[e] - 64ll * e);
  const int32_t *dl = dofs + doff[e];
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  float *Cs = fsm;              // n x noccp
  float *fs = Cs + n * noccp;   // noccp
  float *Cz = fs + noccp;       // n x noccp: imaginary parts (Bloch states, Ci != nullptr)
  for (int k = threadIdx.x; k < n * noccp; k += DEN_NT) {
    const int j = k / noccp, kk = k - j * noccp;
    if (BLOCH) {   // (C + i Ci) exp(i k.R_j) in FP64, then rounded
      double cr = 0.0, ci = 0.0;
      if (kk < nocc) {
        const double ar = C[(int64_t)dl[j] * ldc + kk], ai = Ci[(int64_t)dl[j] * ldc + kk];
        const int c = eshift[doff[e] + j];
        cr = ph.re[c] * ar - ph.im[c] * ai;
        ci = ph.re[c] * ai + ph.im[c] * ar;
      }
      Cs[k] = (float)cr;
      Cz[k] = (float)ci;
    } else {
      Cs[k] = (kk < nocc) ? (float)C[(int64_t)dl[j] * ldc + kk] : 0.0f;
    }
  }
  for (int k = threadIdx.x; k < noccp; k += DEN_NT) fs[k] = (k < nocc) ? (float)f[k] : 0.0f;
  __syncthreads();
  for (int q = qb + threadIdx.x; q < Q; q += DEN_NT) {
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
    // real parts (the only ones at Gamma), then the imaginary parts; at Gamma
    // states 16 at a time while 16 remain, then 8 (each state's sums in the
    // same order either way; the Bloch form measured faster with 8 only)
    for (int part = 0; part < (BLOCH ? 2 : 1); ++part) {
      const float *Cb = part ? Cz : Cs;
      int k0 = 0;
      for (; !BLOCH && k0 + 16 <= noccp; k0 += 16)
        r = density_states<16>(L, pu, pq, ec, nenr, Cb, fs, noccp, k0, r);
      for (; k0 < noccp; k0 += 8) r = density_states<8>(L, pu, pq, ec, nenr, Cb, fs, noccp, k0, r);
    }
    rho[q0 + q] = (double)r;
  }
}

// ---------------------------------------------------------------------------
// K5' (FP32): Vbar_q = w_q b_q^T Hbar_e b_q.  One CTA per element: Hbar_e
// (gathered through the scatter map) and a chunk of 32 basis rows sit in
// shared memory; each thread owns a 4-point x 4-row register tile of
// t_qi = sum_j Hbar_ij b_qj and stores its rows' sum of b_qi t_qi per point;
// the row tiles' sums are then added in a fixed order.
// ---------------------------------------------------------------------------
constexpr int ADJ_NT = 256;
constexpr int ADJ_QB = 32;

template <bool BLOCH>
__global__ void __launch_bounds__(ADJ_NT) k_adjoint_f32(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const double *__restrict__ w, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap,
    const double *__restrict__ Hbar, double *__restrict__ Vbar,
    const int32_t *__restrict__ items, BlochCot bc) {
  extern __shared__ __align__(16) float fsm[];
  // work item: the points [8 c0, 8 c1) of element order[items[3 b]] (clipped
  // to the element's Q points)
  const int e = order[items[3 * blockIdx.x]];
  const int64_t q0 = qoff[e];
  const int Q = (int)(qoff[e + 1] - q0);
  const int qbeg = items[3 * blockIdx.x + 1] * 8;
  const int qend = min(Q, items[3 * blockIdx.x + 2] * 8);
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
  float *part = Bq + ADJ_QB * ldb; // (n4 / 4) x ADJ_QB: each row tile's sum per point
  for (int k = threadIdx.x; k < n4 * n4; k += ADJ_NT) {
    const int i = k / n4, j = k - i * n4;
    float v = 0.0f;
    if (i < n && j < n) {
      const int32_t sl = m[i * n + j];
      v = BLOCH ? (float)cot_entry(Hbar[sl], bc.Hi[sl], bc.eshift[doff[e] + i],
                                   bc.eshift[doff[e] + j], bc.ph)
                : (float)Hbar[sl];
    }
    Hs[k] = v;
  }
  const int nI = n4 / 4;
  const int ntile = (ADJ_QB / 4) * nI;
  for (int qc = qbeg; qc < qend; qc += ADJ_QB) {
    __syncthreads();
    for (int k = threadIdx.x; k < ADJ_QB * n4; k += ADJ_NT) {
      const int qq = k / n4, c = k - qq * n4;
      const int q = qc + qq;
      float b = 0.0f;
      if (q < qend && c < n) {
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
        part[ti * ADJ_QB + 4 * tq + x] = s;
      }
    }
    __syncthreads();
    // the row tiles' sums added in a fixed order (a deterministic result)
    if (threadIdx.x < ADJ_QB && qc + (int)threadIdx.x < qend) {
      float s = 0.0f;
      for (int ti = 0; ti < nI; ++ti) s += part[ti * ADJ_QB + threadIdx.x];
      Vbar[q0 + qc + threadIdx.x] = w[q0 + qc + threadIdx.x] * (double)s;
    }
  }
}

// ---------------------------------------------------------------------------
// K5 enrichment strip on the CUDA cores (elements with n_e <= 128).
// With b = (b_F, b_E) split into the 64 FE functions and the enrichments,
//   b^T Hbar b = b_F^T Hbar_FF b_F + sum_{r in E} b_r g_r,
//   g_r = sum_j B[r][j] b_j,  B[r][j] = Hbar_rj + Hbar_jr (j in F),
// where the FE-FE form is done by sum factorization (k_adjoint_fefe, which
// stores Vbar) and this kernel adds w_q sum_r b_r g_r, one thread per point,
// in FP32 with round to nearest:
//   FE columns:  g_r += sum_(abc) B[r][(abc)] L_a(x) L_b(y) L_c(z), factorized
//                per point (84 multiply-adds per r instead of 128);
//   E columns:   the E-E form is symmetric in (r, s), so only s >= r is kept:
//                Be[s][r] = Hbar_rr (s = r), Hbar_rs + Hbar_sr (s > r).
// Rows r go in register blocks of 8, so each broadcast read of B feeds 8 FMAs.
// ---------------------------------------------------------------------------
constexpr int AS_NT = 256;

template <bool BLOCH>
__global__ void __launch_bounds__(AS_NT) k_adjoint_strip_f32(
    const int32_t *__restrict__ order, const int64_t *__restrict__ qoff,
    const int64_t *__restrict__ qpoff, const float4 *__restrict__ qdat,
    const double *__restrict__ w, const int64_t *__restrict__ doff,
    const int32_t *__restrict__ ecol, const int32_t *__restrict__ aoff,
    const int64_t *__restrict__ toff32, const float *__restrict__ psi,
    const int64_t *__restrict__ soff, const int32_t *__restrict__ smap,
    const int32_t *__restrict__ partoff, const int32_t *__restrict__ part_p,
    const double *__restrict__ Hbar, double *__restrict__ Vbar,
    const int32_t *__restrict__ pitems, BlochCot bc) {
  extern __shared__ float4 sm_as4[];
  // work item: points [qb, Q) of element order[k]
  const int e = order[pitems[3 * blockIdx.x]], tid = threadIdx.x;
  const int qb = pitems[3 * blockIdx.x + 1], qend = pitems[3 * blockIdx.x + 2];
  const int n = (int)(doff[e + 1] - doff[e]);
  const int ne = n - 64;
  if (ne <= 0 || n > 128) return;   // FE-only (Vbar complete) or a tensor-core element
  {  // elements of the slot form are done by k_adjoint_strip_sf
    int pmax = 0;
    for (int k = partoff[e]; k < partoff[e + 1]; ++k) pmax = max(pmax, part_p[k]);
    if (adjoint_sf_fits(aoff[e + 1] - aoff[e], pmax)) return;
  }
  const int ne8 = (ne + 7) & ~7;
  float *Bf = reinterpret_cast<float *>(sm_as4);   // [64][ne8]: B[r][j], j in F
  float *Be = Bf + 64 * ne8;                       // [ne8][ne8]: s >= r half
  float *bE = Be + ne8 * ne8;                      // [ne8][AS_NT]: b_s at each point
  int *ecs = reinterpret_cast<int *>(bE + ne8 * AS_NT);
  const int64_t q0 = qoff[e];
  const int Q = min((int)(qoff[e + 1] - q0), qend);
  const int A = aoff[e + 1] - aoff[e];
  const int32_t *m = smap + soff[e];
  const float *pe = psi + 4 * toff32[e];
  const float4 *qe = qdat + qpoff[e];
  if (tid < ne) ecs[tid] = ecol[(doff[e] - 64ll * e) + tid];
  // element entry (i, j) of the cotangent (the phased real part at a wavevector)
  auto hv = [&](int i, int j) -> double {
    const int32_t sl = m[i * n + j];
    return BLOCH ? cot_entry(Hbar[sl], bc.Hi[sl], bc.eshift[doff[e] + i], bc.eshift[doff[e] + j],
                             bc.ph)
                 : Hbar[sl];
  };
  for (int o = tid; o < 64 * ne8; o += AS_NT) {
    const int j = o / ne8, r = o - j * ne8;
    Bf[o] = r < ne ? (float)(hv(64 + r, j) + hv(j, 64 + r)) : 0.0f;
  }
  for (int o = tid; o < ne8 * ne8; o += AS_NT) {
    const int sr = o / ne8, r = o - sr * ne8;
    float v = 0.0f;
    if (sr < ne && sr > r) v = (float)(hv(64 + r, 64 + sr) + hv(64 + sr, 64 + r));
    else if (sr < ne && sr == r) v = (float)hv(64 + r, 64 + r);
    Be[o] = v;
  }
  __syncthreads();
  for (int t0 = qb; t0 < Q; t0 += AS_NT) {
    const int ql = t0 + tid;
    if (ql >= Q) break;   // no block-wide barrier below
    const float4 x4 = qe[ql];
    float Lx[4], Ly[4], Lz[4], dL[4];
    lagrange3f(x4.x, Lx, dL);
    lagrange3f(x4.y, Ly, dL);
    lagrange3f(x4.z, Lz, dL);
    const float *pq = pe + (int64_t)(ql >> 3) * A * 32 + (ql & 7);
    for (int sr = 0; sr < ne8; ++sr) {   // this thread's own column only
      float b = 0.0f;
      if (sr < ne) {
        const int code = ecs[sr], lv = code & 7;
        const float phi = ((lv & 1) ? 1.0f + x4.x : 1.0f - x4.x) *
                          ((lv & 2) ? 1.0f + x4.y : 1.0f - x4.y) *
                          ((lv & 4) ? 1.0f + x4.z : 1.0f - x4.z);
        b = 0.125f * phi * pq[(code >> 3) * 32];
      }
      bE[sr * AS_NT + tid] = b;
    }
    float acc = 0.0f;
    for (int r0 = 0; r0 < ne8; r0 += 8) {
      float g[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) g[k] = 0.0f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float tb[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) tb[k] = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float ta[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) ta[k] = 0.0f;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float4 *bp = reinterpret_cast<const float4 *>(Bf + (a + 4 * b + 16 * c) * ne8 + r0);
            const float4 u = bp[0], v = bp[1];
            ta[0] = fmaf(Lx[a], u.x, ta[0]);
            ta[1] = fmaf(Lx[a], u.y, ta[1]);
            ta[2] = fmaf(Lx[a], u.z, ta[2]);
            ta[3] = fmaf(Lx[a], u.w, ta[3]);
            ta[4] = fmaf(Lx[a], v.x, ta[4]);
            ta[5] = fmaf(Lx[a], v.y, ta[5]);
            ta[6] = fmaf(Lx[a], v.z, ta[6]);
            ta[7] = fmaf(Lx[a], v.w, ta[7]);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) tb[k] = fmaf(Ly[b], ta[k], tb[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = fmaf(Lz[c], tb[k], g[k]);
      }
      for (int sr = r0; sr < ne8; ++sr) {
        const float bs = bE[sr * AS_NT + tid];
        const float4 *bp = reinterpret_cast<const float4 *>(Be + sr * ne8 + r0);
        const float4 u = bp[0], v = bp[1];
        g[0] = fmaf(u.x, bs, g[0]);
        g[1] = fmaf(u.y, bs, g[1]);
        g[2] = fmaf(u.z, bs, g[2]);
        g[3] = fmaf(u.w, bs, g[3]);
        g[4] = fmaf(v.x, bs, g[4]);
        g[5] = fmaf(v.y, bs, g[5]);
        g[6] = fmaf(v.z, bs, g[6]);
        g[7] = fmaf(v.w, bs, g[7]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) acc = fmaf(bE[(r0 + k) * AS_NT + tid], g[k], acc);
    }
    Vbar[q0 + ql] += w[q0 + ql] * (double)acc;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
pufe_status launch_tabulate_f32(pufe_ctx *ctx, cudaStream_t st) {
  if (ctx->psi32_len == 0) return PUFE_OK;
  auto &D = ctx->d;
  if (ctx->n_tblk <= 0) return PUFE_OK;
  k_tabulate_f32<<<(unsigned)ctx->n_tblk, TAB_NT, 0, st>>>(
      D.qpoff, D.qdat, D.aoff, D.alist, D.toff32, D.orbf, D.eorig, (float)ctx->a[0],
      (float)ctx->a[1], (float)ctx->a[2], (float)ctx->h[0], (float)ctx->h[1], (float)ctx->h[2],
      D.tblk, (int)ctx->nelem, D.psi32);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

// H/S assembly on the mixed path: H = 0 and S = the constant FE-FE overlap,
// then the FE-FE blocks of H (kinetic constants + sum-factorized V term), the
// enrichment strips (tensor cores for n_e > 128, CUDA cores otherwise) and the
// E-E block of S, all adding into H and S; `vscratch` receives the FP32 copy
// of V that the tensor-core kernel reads (nq_pad floats).
static pufe_status run_assemble_tc(pufe_ctx *ctx, const double *V, int what, double *H,
                                   double *S, float *vscratch, cudaStream_t st) {
  auto &D = ctx->d;
  if (!ctx->fe_exact)
    return fail(PUFE_EINVAL,
                "PUFE_TF32X3 needs every (sub)cell rule to have >= 4 points per axis");
  if (ctx->max_basis > 256) return fail(PUFE_EINVAL, "PUFE_TF32X3 supports n_e <= 256");
  const int amax = std::max(1, ctx->max_alpha);
  const int inb = ((amax * 4 * WS_KC * 4 + WS_KC * 128 + WS_KC * 4) + 127) & ~127;
  const size_t sm256 = assemble_smem(inb);
  const int nbig = ctx->n_big;
  const int nsmall = (int)ctx->nelem - nbig;
  if (nbig > 0 && sm256 > 227 * 1024)
    return fail(PUFE_EINVAL, "too many enrichments per element for TF32X3");
  // H = 0 and S = the constant FE-FE overlap; then the strip kernels on the
  // caller's stream and, on the context's side stream, the FE-FE kernel (V
  // term and kinetic constants of H) and the E-E kernel of S, concurrently
  // (all of them only add into H and S)
  if (ctx->max_part_p > 16) return fail(PUFE_EINVAL, "rule with more than 16 points per axis");
  const bool prof = ctx->prof;
  auto mark = [&](int i, cudaStream_t s) -> pufe_status {
    if (prof) PUFE_CUDA_TRY(cudaEventRecord(ctx->pev[i], s));
    return PUFE_OK;
  };
  if (prof)
    for (bool &r : ctx->prof_ran) r = false;
  if (pufe_status e = mark(0, st)) return e;
  if (prof) ctx->prof_ran[0] = true;
  const size_t bytes = (size_t)ctx->nnz * sizeof(double);
  if (what & PUFE_WANT_H) PUFE_CUDA_TRY(cudaMemsetAsync(H, 0, bytes, st));
  if (what & PUFE_WANT_S) PUFE_CUDA_TRY(cudaMemcpyAsync(S, D.S0, bytes, cudaMemcpyDeviceToDevice, st));
  PUFE_CUDA_TRY(cudaEventRecord(D.ev_fork, st));
  // the strip kernels go first, so that their CTAs take their share of every
  // SM; the side stream's kernels are small enough to run beside them
  if (nbig > 0) {
    // every entry the tensor-core kernel reads is rewritten (zeros on padding)
    k_pack_v<<<(unsigned)nbig, 256, 0, st>>>(D.order, D.qoff, D.qpoff,
                                             (what & PUFE_WANT_H) ? V : nullptr, vscratch);
    PUFE_CUDA_TRY(cudaGetLastError());
    const float sx = (float)(2.0 / ctx->h[0]), sy = (float)(2.0 / ctx->h[1]),
                sz = (float)(2.0 / ctx->h[2]);
    int nsm = 0;
    PUFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    PUFE_CUDA_TRY(cudaFuncSetAttribute(k_assemble_tc,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm256));
    if (pufe_status e = mark(6, st)) return e;
    k_assemble_tc<<<std::min(ctx->n_titems, nsm), WS_NT, sm256, st>>>(
        D.order, D.qoff, D.qpoff, D.ptab, vscratch, D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
        D.soff, D.smap, sx, sy, sz, D.titems, ctx->n_titems, amax, inb, what, H, S, D.err);
    PUFE_CUDA_TRY(cudaGetLastError());
    if (pufe_status e = mark(7, st)) return e;
    if (prof) ctx->prof_ran[3] = true;
  }
  if (pufe_status e = mark(8, st)) return e;
  pufe_status e1 = launch_strip_sf(ctx, (what & PUFE_WANT_H) ? V : nullptr, what, H, S, nbig, nsmall, st);
  if (e1 != PUFE_OK) return e1;
  if (pufe_status e = mark(9, st)) return e;
  if (prof) ctx->prof_ran[4] = nsmall > 0;
  // the E-E kernels of S on the side stream; the FE-FE kernel after the strip
  // on the caller's stream when no tensor-core tile runs there, else on the
  // side stream before the E-E kernels (measured: 12^3 rocksalt step 0.559 ->
  // 0.543 ms with it on the caller's stream; the CsCl-like cell, whose
  // caller's stream also carries the tensor-core tile, 1.71 -> 1.76 ms)
  PUFE_CUDA_TRY(cudaStreamWaitEvent(D.side, D.ev_fork, 0));
  if (what & PUFE_WANT_H) {
    const cudaStream_t sf = nbig > 0 ? D.side : st;
    if (pufe_status e = mark(2, sf)) return e;
    pufe_status e0 = launch_fefe(ctx, V, H, sf);
    if (e0 != PUFE_OK) return e0;
    if (pufe_status e = mark(3, sf)) return e;
    if (prof) ctx->prof_ran[1] = true;
  }
  if (what & PUFE_WANT_S) {
    if (pufe_status e = mark(4, D.side)) return e;
    pufe_status e0 = launch_see(ctx, nullptr, S, nullptr, D.side);
    if (e0 != PUFE_OK) return e0;
    if (pufe_status e = mark(5, D.side)) return e;
    if (prof) ctx->prof_ran[2] = true;
  }
  PUFE_CUDA_TRY(cudaEventRecord(D.ev_join, D.side));
  PUFE_CUDA_TRY(cudaStreamWaitEvent(st, D.ev_join, 0));
  if (pufe_status e = mark(1, st)) return e;
  return PUFE_OK;
}

pufe_status launch_wait_probe(pufe_ctx *ctx, uint64_t wait_ns, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(wait_ns, ctx->d.err);
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status profile_enable(pufe_ctx *ctx, bool on) {
  if (on && !ctx->pev[0])
    for (auto &ev : ctx->pev) PUFE_CUDA_TRY(cudaEventCreate(&ev));
  ctx->prof = on;
  return PUFE_OK;
}

pufe_status profile_read(pufe_ctx *ctx, double ms[5]) {
  for (int k = 0; k < 5; ++k) ms[k] = 0.0;
  if (!ctx->pev[0] || !ctx->prof_ran[0]) return fail(PUFE_ESTATE, "no instrumented call to read");
  PUFE_CUDA_TRY(cudaEventSynchronize(ctx->pev[1]));
  for (int k = 0; k < 5; ++k) {
    if (!ctx->prof_ran[k]) continue;
    float t = 0.0f;
    PUFE_CUDA_TRY(cudaEventElapsedTime(&t, ctx->pev[2 * k], ctx->pev[2 * k + 1]));
    ms[k] = t;
  }
  return PUFE_OK;
}

pufe_status launch_assemble_tc(pufe_ctx *ctx, const double *V, int what, double *H, double *S,
                               cudaStream_t st) {
  return run_assemble_tc(ctx, V, what, H, S, ctx->d.vpad, st);
}

pufe_status launch_density_tc(pufe_ctx *ctx, const double *C, int64_t ldc, const double *f,
                              int nocc, double *rho, cudaStream_t st, const double *Ci,
                              const PhaseTab *ph) {
  auto &D = ctx->d;
  const int noccp = (nocc + 7) & ~7;
  const size_t sm = ((size_t)ctx->max_basis * noccp * (Ci ? 2 : 1) + noccp) * sizeof(float);
  if (sm > 227 * 1024) return fail(PUFE_EINVAL, "density: basis x states beyond shared memory");
  if (Ci && !ph) return fail(PUFE_EINVAL, "internal: Bloch density without phases");
  auto kern = Ci ? k_density_f32<true> : k_density_f32<false>;
  PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  if (ctx->n_pitems <= 0) return PUFE_OK;
  kern<<<(unsigned)ctx->n_pitems, DEN_NT, sm, st>>>(
      D.order, D.qoff, D.qpoff, D.qdat, D.doff, D.dofs, D.ecol, D.aoff, D.toff32, D.psi32, C,
      ldc, f, nocc, noccp, rho, D.pitems, Ci, D.eshift, ph ? *ph : PhaseTab{});
  PUFE_CUDA_TRY(cudaGetLastError());
  return PUFE_OK;
}

pufe_status launch_adjoint_tc(pufe_ctx *ctx, const double *Hbar, double *Vbar, cudaStream_t st,
                              const BlochCot *bcp) {
  auto &D = ctx->d;
  const BlochCot bc = bcp ? *bcp : BlochCot{nullptr, nullptr, PhaseTab{}};
  const int nbig = ctx->n_big;
  if (nbig > 0) {  // n_e > 128: FP32 CUDA-core kernel
    const int n4 = (ctx->max_basis + 3) & ~3;
    const int ldb = n4 + 36;
    const size_t sm = ((size_t)n4 * n4 + (size_t)ADJ_QB * ldb + (size_t)(n4 / 4) * ADJ_QB) *
                      sizeof(float);
    if (sm > 227 * 1024) return fail(PUFE_EINVAL, "n_e too large for the FP32 adjoint kernel");
    auto kern = bc.Hi ? k_adjoint_f32<true> : k_adjoint_f32<false>;
    PUFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    kern<<<ctx->n_titems, ADJ_NT, sm, st>>>(D.order, D.qoff, D.qpoff, D.qdat, D.w,
                                                     D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
                                                     D.soff, D.smap, Hbar, Vbar, D.titems,
                                                     bc);
    PUFE_CUDA_TRY(cudaGetLastError());
  }
  const int nsmall = (int)ctx->nelem - nbig;
  if (nsmall > 0) {  // n_e <= 128: FE-FE by sum factorization, then the enrichment strip
    int ne8 = 8;
    for (int64_t k = nbig; k < ctx->nelem; ++k)
      ne8 = std::max(ne8, (ctx->n_e[ctx->order[k]] - 64 + 7) & ~7);
    const size_t sm = ((size_t)64 * ne8 + (size_t)ne8 * ne8 + (size_t)ne8 * AS_NT + ne8) * 4;
    if (sm > 227 * 1024) return fail(PUFE_EINVAL, "n_e too large for the strip adjoint");
    pufe_status e0 = launch_adjoint_fefe(ctx, Hbar, Vbar, nbig, nsmall, st, bc);
    if (e0 != PUFE_OK) return e0;
    // the slot form where it fits (all elements of the usual rules), the
    // direct per-point form for the rest
    pufe_status e1 = launch_adjoint_strip_sf(ctx, Hbar, Vbar, nbig, nsmall, st, bc);
    if (e1 != PUFE_OK) return e1;
    if (!ctx->adj_sf_all) {
      auto kern = bc.Hi ? k_adjoint_strip_f32<true> : k_adjoint_strip_f32<false>;
      PUFE_CUDA_TRY(
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      kern<<<(unsigned)ctx->n_pitems, AS_NT, sm, st>>>(
          D.order, D.qoff, D.qpoff, D.qdat, D.w, D.doff, D.ecol, D.aoff, D.toff32, D.psi32,
          D.soff, D.smap, D.partoff, D.part_p, Hbar, Vbar, D.pitems, bc);
      PUFE_CUDA_TRY(cudaGetLastError());
    }
  }
  return PUFE_OK;
}

}  // namespace pufe

// ---------------------------------------------------------------------------
// Allocation-free variant of the TF32X3 assembly.
//
// The assembly kernel reads an FP32 copy of V laid out on the padded point
// list; pufe_assemble_HS keeps that copy in memory the context allocated.
// This variant keeps it in the file-scope array below instead, so a call
// needs no device allocation of any kind.  The array holds at most
// PUFE_STATIC_MAX_POINTS values on every device that loads the library (it
// stays resident until the process exits); larger contexts are rejected.
// The device address of the array is looked up once per device with
// cudaGetSymbolAddress (the host-side symbol is only a stand-in) on the
// first call made on that device; it stays valid while that device's primary
// context lives (a cudaDeviceReset ends it).
// ---------------------------------------------------------------------------
#define PUFE_STATIC_MAX_POINTS (4 * 1024 * 1024)
static __device__ __align__(256) float g_vpad_static[PUFE_STATIC_MAX_POINTS];

namespace pufe {
namespace {
std::mutex g_static_mu;
float *g_static_ptr[128] = {nullptr};
}  // namespace

static pufe_status static_scratch(int device, float **out) {
  if (device < 0 || device >= 128) return fail(PUFE_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_vpad_static);  // the ctx device is current
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_vpad_static)");
    g_static_ptr[device] = static_cast<float *>(p);
  }
  *out = g_static_ptr[device];
  return PUFE_OK;
}

pufe_status launch_assemble_tc_static(pufe_ctx *ctx, const double *V, int what, double *H,
                                      double *S, cudaStream_t st) {
  // the array is indexed by the padded point offsets of the n_e > 128
  // elements (the only ones whose V it carries)
  if (ctx->big_pad_end > PUFE_STATIC_MAX_POINTS)
    return fail(PUFE_EINVAL, "pufe_assemble_HS_static: the elements with more than 128 basis "
                             "functions end at padded quadrature point " +
                                 std::to_string(ctx->big_pad_end) +
                                 "; the static scratch holds " +
                                 std::to_string(PUFE_STATIC_MAX_POINTS));
  float *vs = nullptr;
  if (pufe_status e0 = static_scratch(ctx->device, &vs)) return e0;
  return run_assemble_tc(ctx, V, what, H, S, vs, st);
}

}  // namespace pufe
