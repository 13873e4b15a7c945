// Restart product U_k = U Q' (Eq. 3.5) of an FP32 basis on the fifth-generation
// tensor cores of sm_103a (tcgen05.mma, accumulators in tensor memory).
//
// Split-BF16: an FP32 value u is the exact sum u1 + u2 + u3 of three bf16
// numbers (u1 = bf16(u), u2 = bf16(u - u1), u3 = bf16(u - u1 - u2); each
// remainder is exact in FP32); Q' is split the same way on the host.  The
// product keeps the six terms u_i q_j with i + j <= 4 (the dropped ones are
// below 2^-32 |u| |q|); every bf16 x bf16 product is exact and the sums are
// FP32 in tensor memory, so the result has FP32-class accuracy.
//
// One CTA (256 threads) owns tiles of 128 rows; per tile the K dimension
// (the nin input columns, padded to kKc) streams through two shared-memory
// stages of 32 columns: all threads load and split a stage (FP32 loads,
// coalesced along the rows, issued one stage ahead into registers) into the
// canonical K-major no-swizzle layout,
// thread 0 issues 2 x 6 MMAs of 128 x N x 16 on it and commits them to the
// stage's mbarrier, which the next load of that stage waits for.  The
// epilogue reads the 128 x N FP32 accumulator with tcgen05.ld (warps 0-3 and
// 4-7 take alternate 16-column groups of their lane quarter) and writes the
// outputs; every read of a tile's rows precedes its writes, so the product
// may be formed in place.  All waits are bounded (RKS_FLAG_TIMEOUT).

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rks_impl.h"

namespace rks {

namespace {

constexpr int kM = 128;           // rows per tile (MMA M)
constexpr int kKc = 32;           // input columns per stage (two MMA K-steps)
constexpr int kThreads = 256;
constexpr int kStageSplit = kM * kKc * 2;   // bytes of one split of one stage
constexpr int kStage = 3 * kStageSplit;
constexpr int kTmemCols = 64;

// Byte offset of element (r, k) of a K-major, no-swizzle tile with `rows`
// rows: K sub-tiles of 16, each of rows/8 groups (stride SBO = 256 B) of two
// 8 x 16-byte core matrices along K (stride LBO = 128 B).
__host__ __device__ inline uint32_t canon_off(int r, int k, int rows) {
  return (uint32_t)((k >> 4) * rows * 32 + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// descriptor version 1 (bits 46-48), no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for the completion of the mbarrier phase with this parity.
__device__ bool mbar_wait(uint32_t mbar, uint32_t parity, int* flag) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000ll) {
      atomicOr(flag, RKS_FLAG_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t bf16_bits(__nv_bfloat16 h) { return (uint32_t)__bfloat16_as_ushort(h); }

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The six split products (i, j) with i + j <= 4, splits numbered 1..3 (0..2 here).
__host__ __device__ constexpr int pair_a(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }
__host__ __device__ constexpr int pair_b(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }

// out[i, o] = sum_l in[i, l] Q'[l, o] for i < n, o < nout; then, when mvsrc
// is given, mvdst[i] = mvsrc[i].  bimg: the three bf16 splits of Q' (Kp x N,
// zero padded) in the canonical layout, split j at byte j * Kp * N * 2.
__global__ void __launch_bounds__(kThreads, 3) k_tc_restart_f32(int64_t n, const float* in, float* out, int64_t ldu,
                                                                int nin, int Kp, int N, int nout,
                                                                const uint4* __restrict__ bimg, const float* mvsrc,
                                                                float* mvdst, int* flag) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bbytes = 3 * Kp * N * 2;
  uint8_t* sB = smem;
  uint8_t* sA = smem + ((bbytes + 1023) & ~1023);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sA + 2 * kStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);

  for (int t = tid; t < bbytes / 16; t += kThreads) reinterpret_cast<uint4*>(sB)[t] = bimg[t];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < 3; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + s)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_bf16(N);
  const uint32_t sA32 = smem_u32(sA), sB32 = smem_u32(sB);
  const int nk = Kp / kKc;
  const int64_t ntiles = (n + kM - 1) / kM;
  int g = 0;                 // stages filled so far (all tiles)
  uint32_t dpar = 0;         // parity of the accumulator-done barrier
  bool ok = true;
  const int r = tid & (kM - 1), kh = tid >> 7;   // loader: row, half of the stage's 32 columns

  // the 16 values (one row, half a stage) that this thread loads for stage kc of a tile
  auto load16 = [&](int64_t tile, int kc, float* v) {
    const int64_t i = tile * kM + r;
    const int l0 = kc * kKc + kh * 16;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int l = l0 + u;
      v[u] = (tile < ntiles && i < n && l < nin) ? in[i + (int64_t)l * ldu] : 0.f;
    }
  };
  // loads run two stages ahead of the split (three register stages): one
  // stage of work is shorter than the DRAM latency
  auto next_step = [&](int64_t& t, int& k) {
    if (++k == nk) { k = 0; t += gridDim.x; }
  };
  float v[16], vn[16], vnn[16];
  int64_t pt = blockIdx.x;
  int pk = 0;
  load16(pt, pk, v);
  next_step(pt, pk);
  load16(pt, pk, vn);
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    for (int kc = 0; kc < nk && ok; ++kc, ++g) {
      const int s = g & 1;
      next_step(pt, pk);
      load16(pt, pk, vnn);
      if (g >= 2) ok = mbar_wait(smem_u32(mbar + s), (uint32_t)(((g - 2) >> 1) & 1), flag);
      ok = __syncthreads_and(ok);
      if (!ok) break;
      uint8_t* st = sA + s * kStage;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t w[3][4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          uint32_t p[3][2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float x = v[h * 8 + u + e];
            const __nv_bfloat16 a = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(a);
            const __nv_bfloat16 b = __float2bfloat16_rn(r1);
            const __nv_bfloat16 c = __float2bfloat16_rn(r1 - __bfloat162float(b));
            p[0][e] = bf16_bits(a);
            p[1][e] = bf16_bits(b);
            p[2][e] = bf16_bits(c);
          }
#pragma unroll
          for (int q = 0; q < 3; ++q) w[q][u >> 1] = p[q][0] | (p[q][1] << 16);
        }
        const uint32_t off = canon_off(r, kh * 16 + h * 8, kM);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          *reinterpret_cast<uint4*>(st + q * kStageSplit + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        fence_after();
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const int ks = kc * 2 + kk;   // K-step of 16 within the padded K
#pragma unroll
          for (int pr = 0; pr < 6; ++pr) {
            const uint64_t a = sdesc(sA32 + s * kStage + pair_a(pr) * kStageSplit + kk * kM * 32);
            const uint64_t b = sdesc(sB32 + pair_b(pr) * Kp * N * 2 + ks * N * 32);
            mma_bf16(tmem, a, b, idesc, (kc | kk | pr) ? 1u : 0u);
          }
        }
        mma_commit(smem_u32(mbar + s));
        if (kc == nk - 1) mma_commit(smem_u32(mbar + 2));
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        v[u] = vn[u];
        vn[u] = vnn[u];
      }
    }
    if (!ok) break;
    // epilogue
    ok = mbar_wait(smem_u32(mbar + 2), dpar, flag);
    dpar ^= 1u;
    ok = __syncthreads_and(ok);
    if (!ok) break;
    fence_after();
    const int q4 = warp & 3;
    const int64_t ir = tile * kM + q4 * 32 + lane;
    float mv = 0.f;
    if (mvsrc && warp < 4 && ir < n) mv = mvsrc[ir];
    for (int cg = warp >> 2; cg < N / 16; cg += 2) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cg * 16), acc);
      if (ir < n) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int o = cg * 16 + j;
          if (o < nout) out[ir + (int64_t)o * ldu] = acc[j];
        }
      }
    }
    if (mvsrc && warp < 4 && ir < n) mvdst[ir] = mv;
    fence_before();
    __syncthreads();   // accumulator read before the next tile's first MMA
  }
  // Every issued MMA has completed unless a wait gave up; then thread 0 waits
  // (bounded again) for the last commit of each barrier before the tensor
  // memory is released.
  if (!ok && tid == 0) {
    const int c0 = (g + 1) / 2, c1 = g / 2;      // commits made to the two stage barriers
    if (c0 > 0) (void)mbar_wait(smem_u32(mbar + 0), (uint32_t)((c0 - 1) & 1), flag);
    if (c1 > 0) (void)mbar_wait(smem_u32(mbar + 1), (uint32_t)((c1 - 1) & 1), flag);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// Double-float basis: exact split products (Ozaki-type) on the tensor cores
// ---------------------------------------------------------------------------
//
// A DF value v = hi + lo of row i is written, relative to the row scale 2^e_i
// (|v| < 2^(e_i - 1) for every input column), as the 47-bit fixed-point
// integer V = round(v 2^(48 - e_i)) = sum_s d_s 2^(42 - 7s), a signed top
// digit d_0 (|d_0| <= 32) and six 7-bit digits (0..127), all exact in bf16;
// Q' likewise per column with scale 2^f_o (digits c_t, built on the host).
// Then
//   sum_l v_l q_l = 2^(e_i + f_o - 12) sum_g 2^(-7g) G_g,
//   G_g = sum_{s + t = g} sum_l d_s(i, l) c_t(l, o),
// with integer G_g.  The 34 digit pairs with s + t <= 7 go to 8 accumulators
// (8 x N tensor-memory columns; the dropped pairs are below 5 * 2^-51 of
// the scale).  For K <= 192 every group of weight above 2^-35 stays below
// 2^24, so the bf16 MMAs with FP32 accumulation in tensor memory sum it
// exactly; a lighter group may round by a unit or two, far below 2^-48.
// The epilogue combines the groups in DF.  K streams through two shared-
// memory stages of one K-step (16 input columns x 7 digit slices); Q'
// (7 slices, all K) stays resident.

constexpr int kDfDigits = 7;
constexpr int kDfThreads = 512;
constexpr int kDfGroups = 8;
constexpr int kDfStepSplit = kM * 16 * 2;                 // one digit slice of one K-step
constexpr int kDfStage = kDfDigits * kDfStepSplit;        // 28 KB

// Largest biased exponent of the hi parts of row i over the nin columns, each
// column taken times 2^pexp[l] (its power-of-two scale; zero entries skipped).
__global__ void k_row_exp(int64_t n, const float2* __restrict__ in, int64_t ldu, int nin,
                          const int* __restrict__ pexp, int* __restrict__ rexp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int em = -100000;
#pragma unroll 8
    for (int l = 0; l < nin; ++l) {
      const int E = (int)((__float_as_uint(in[i + (int64_t)l * ldu].x) >> 23) & 0xFFu);
      if (E != 0) em = max(em, E + pexp[l]);
    }
    rexp[i] = em;
  }
}

// bf16 bits of a small integer 0 <= d < 256 on the full-rate pipes: the
// float 2^23 + d minus 2^23 is d exactly, and its low 16 bits are zero.
__device__ __forceinline__ uint32_t small_bf16(int d) {
  return __float_as_uint(__int_as_float(0x4B000000 | d) - 8388608.0f) >> 16;
}

// round(x 2^(48 - e)) with e = emax - 125, from the bits of x (|result| <= 2^47 + 1);
// a column scale 2^p is applied by passing emax - p
__device__ __forceinline__ int64_t fixed48(float x, int emax) {
  const uint32_t b = __float_as_uint(x);
  int E = (int)((b >> 23) & 0xFFu);
  uint32_t m = b & 0x7FFFFFu;
  if (E == 0) E = 1; else m |= 0x800000u;
  const int sh = E - emax + 23;                  // E - 102 - e
  int64_t V;
  if (sh >= 0) V = (int64_t)m << min(sh, 40);   // sh <= 23 except for an all-zero row (m = 0)
  else if (sh > -26) V = (int64_t)((m + (1u << (-sh - 1))) >> -sh);
  else V = 0;
  return (b >> 31) ? -V : V;
}

// out[i, o] = sum_l in[i, l] 2^pexp[l] Q'[l, o] (DF) for i < n, o < nout;
// then, when mvsrc is given, mvdst[i] = mvsrc[i].  bimg: the digit slices of
// Q' (Kp x N, canonical layout, slice t at byte t * Kp * N * 2); fexp[o] =
// f_o; rexp[i] from k_row_exp.  Every read of a tile's rows precedes its
// writes (in place).
//
// Warp roles: warps 0..15 (kDfThreads threads) load and split the digits of
// one K-step into a shared-memory stage and run the epilogue; warp 16 issues
// the MMAs.  Per stage s: full[s] (the splitters arrive once the digits are
// stored) and empty[s] (the MMA commit arrives once they are consumed); per
// tile: done (accumulators complete) and tfree (the epilogue has read them).
// The split of step g + 1 thus overlaps the MMA issue of step g.  Every wait
// is bounded (mbar_wait); the splitters agree on the outcome at their named
// barrier, so a timeout ends every role's loop.
__device__ __forceinline__ bool splitters_and(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred P, Q;\n\tsetp.ne.u32 P, %1, 0;\n\tbar.red.and.pred Q, 1, %2, P;\n\t"
      "selp.u32 %0, 1, 0, Q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(kDfThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

constexpr int kDfAllThreads = kDfThreads + 32;

__global__ void __launch_bounds__(kDfAllThreads, 1) k_tc_restart_df(int64_t n, const float2* in, float2* out,
                                                                    int64_t ldu, int nin, int Kp, int N, int nout,
                                                                    const uint4* __restrict__ bimg,
                                                                    const int* __restrict__ fexp,
                                                                    const int* __restrict__ pexp,
                                                                    const int* __restrict__ rexp,
                                                                    const float2* mvsrc, float2* mvdst, int tcols,
                                                                    int* flag) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bbytes = kDfDigits * Kp * N * 2;
  uint8_t* sB = smem;
  uint8_t* sA = smem + ((bbytes + 1023) & ~1023);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sA + 2 * kDfStage);   // full[2], empty[2], done, tfree
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 6);
  int* sp = reinterpret_cast<int*>(mbar + 7);            // column power-of-two scales (Kp)
  const uint32_t full0 = smem_u32(mbar + 0), empty0 = smem_u32(mbar + 2);
  const uint32_t done_b = smem_u32(mbar + 4), tfree_b = smem_u32(mbar + 5);

  for (int t = tid; t < bbytes / 16; t += kDfAllThreads) reinterpret_cast<uint4*>(sB)[t] = bimg[t];
  for (int t = tid; t < Kp; t += kDfAllThreads) sp[t] = t < nin ? pexp[t] : 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < 6; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + s)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const int nk = Kp / 16;
  const int64_t ntiles = (n + kM - 1) / kM;
  bool ok = true;

  if (warp == kDfThreads / 32) {
    // ---- MMA issuer (lane 0 of warp 16)
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(N);
      const uint32_t sA32 = smem_u32(sA), sB32 = smem_u32(sB);
      int g = 0, tcount = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tcount) {
        if (tcount > 0) {   // the epilogue of the previous tile has read the accumulators
          ok = mbar_wait(tfree_b, (uint32_t)((tcount - 1) & 1), flag);
          if (!ok) break;
          fence_after();
        }
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int s = g & 1;
          ok = mbar_wait(full0 + 8u * s, (uint32_t)((g >> 1) & 1), flag);
          if (!ok) break;
          fence_after();
          const bool first = kc == 0;
#pragma unroll
          for (int gg = 0; gg < kDfGroups; ++gg)
#pragma unroll
            for (int sa = gg < kDfDigits ? 0 : gg - kDfDigits + 1; sa <= gg && sa < kDfDigits; ++sa) {
              const int tb = gg - sa;
              const int sa0 = gg < kDfDigits ? 0 : gg - kDfDigits + 1;   // first pair of the group
              const uint64_t a = sdesc(sA32 + s * kDfStage + sa * kDfStepSplit);
              const uint64_t b = sdesc(sB32 + tb * Kp * N * 2 + kc * N * 32);
              mma_bf16(tmem + (uint32_t)(gg * N), a, b, idesc, (first && sa == sa0) ? 0u : 1u);
            }
          mma_commit(empty0 + 8u * s);
          if (kc == nk - 1) mma_commit(done_b);
        }
      }
      // every issued MMA has completed before the accumulators are freed
      if (g > 0) (void)mbar_wait(empty0 + 8u * ((g - 1) & 1), (uint32_t)(((g - 1) >> 1) & 1), flag);
      if (g > 1) (void)mbar_wait(empty0 + 8u * ((g - 2) & 1), (uint32_t)(((g - 2) >> 1) & 1), flag);
    }
    __syncwarp();
  } else {
    // ---- splitters (warps 0..15) and the epilogue
    int g = 0;                 // stages filled so far (all tiles)
    uint32_t dpar = 0;         // parity of the accumulator-done barrier
    const int r = tid & (kM - 1), kq = tid >> 7;   // loader: row, quarter of the K-step's 16 columns
    auto load4 = [&](int64_t tile, int kc, float2* v) {
      const int64_t i = tile * kM + r;
      const int l0 = kc * 16 + kq * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int l = l0 + u;
        v[u] = (tile < ntiles && i < n && l < nin) ? in[i + (int64_t)l * ldu] : make_float2(0.f, 0.f);
      }
    };
    auto next_step = [&](int64_t& t, int& k) {
      if (++k == nk) { k = 0; t += gridDim.x; }
    };
    float2 v[4], vn[4];   // the next K-step's values are loaded during this one's split
    int64_t pt = blockIdx.x;
    int pk = 0;
    load4(pt, pk, v);
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t irow = tile * kM + r;
      const int emax = irow < n ? rexp[irow] : 0;
      for (int kc = 0; kc < nk && ok; ++kc, ++g) {
        const int s = g & 1;
        next_step(pt, pk);
        load4(pt, pk, vn);
        if (g >= 2) ok = mbar_wait(empty0 + 8u * s, (uint32_t)(((g - 2) >> 1) & 1), flag);
        ok = splitters_and(ok);
        if (!ok) break;
        // digits of 4 values of one row
        uint32_t w[kDfDigits][2];
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          uint32_t pk2[kDfDigits][2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float2 x = v[u + e];
            const int ep = emax - sp[kc * 16 + kq * 4 + u + e];
            const int64_t V = fixed48(x.x, ep) + fixed48(x.y, ep);
            // digits from two 32-bit halves: bits 21..47 (signed) and 0..20
            const int vh = (int)(V >> 21);
            const int vl = (int)(V & 0x1FFFFF);
            const int d0 = vh >> 21;                                   // -32 .. 32
            pk2[0][e] = __float_as_uint(__int_as_float(0x4B000000 | (d0 + 128)) - 8388736.0f) >> 16;
            pk2[1][e] = small_bf16((vh >> 14) & 127);
            pk2[2][e] = small_bf16((vh >> 7) & 127);
            pk2[3][e] = small_bf16(vh & 127);
            pk2[4][e] = small_bf16(vl >> 14);
            pk2[5][e] = small_bf16((vl >> 7) & 127);
            pk2[6][e] = small_bf16(vl & 127);
          }
#pragma unroll
          for (int q = 0; q < kDfDigits; ++q) w[q][u >> 1] = pk2[q][0] | (pk2[q][1] << 16);
        }
        uint8_t* st = sA + s * kDfStage;
        const uint32_t off = canon_off(r, kq * 4, kM);
#pragma unroll
        for (int q = 0; q < kDfDigits; ++q)
          *reinterpret_cast<uint2*>(st + q * kDfStepSplit + off) = make_uint2(w[q][0], w[q][1]);
        fence_async_smem();
        asm volatile("bar.sync 1, %0;" ::"n"(kDfThreads) : "memory");
        if (tid == 0) mbar_arrive(full0 + 8u * s);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = vn[u];
      }
      if (!ok) break;
      // epilogue: sum_g 2^(-7g) G_g in DF, times 2^(e_i + f_o - 12)
      ok = mbar_wait(done_b, dpar, flag);
      dpar ^= 1u;
      ok = splitters_and(ok);
      if (!ok) break;
      fence_after();
      const int q4 = warp & 3;
      const int64_t ir = tile * kM + q4 * 32 + lane;
      const int er = ir < n ? rexp[ir] - 125 : 0;
      float2 mv = make_float2(0.f, 0.f);
      if (mvsrc && warp < 4 && ir < n) mv = mvsrc[ir];
      for (int cg = warp >> 2; cg < N / 16; cg += kDfThreads / 128) {
        float hs[16], ls[16];
        {
          float gv[16];
          tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((kDfGroups - 1) * N + cg * 16), gv);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) { hs[jj] = gv[jj]; ls[jj] = 0.f; }
        }
        for (int gg = kDfGroups - 2; gg >= 0; --gg) {
          float gv[16];
          tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(gg * N + cg * 16), gv);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const float sh = hs[jj] * 0.0078125f, sl = ls[jj] * 0.0078125f;   // exact scaling by 2^-7
            float s2, e2;
            two_sum_f(gv[jj], sh, s2, e2);
            hs[jj] = s2;
            ls[jj] = e2 + sl;
          }
        }
        if (ir < n) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int o = cg * 16 + jj;
            if (o < nout) {
              const int sc = er + fexp[o] - 12;
              float h, l;
              two_sum_f(hs[jj], ls[jj], h, l);
              out[ir + (int64_t)o * ldu] = make_float2(ldexpf(h, sc), ldexpf(l, sc));
            }
          }
        }
      }
      if (mvsrc && warp < 4 && ir < n) mvdst[ir] = mv;
      fence_before();
      asm volatile("bar.sync 1, %0;" ::"n"(kDfThreads) : "memory");
      if (tid == 0) mbar_arrive(tfree_b);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

uint16_t host_bf16(float x) {   // round to nearest even (finite inputs)
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

double host_bf16_value(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

}  // namespace

bool tc_restart_supported(int nin, int nout) { return nin >= 1 && nin <= 256 && nout >= 1 && nout <= 64; }

size_t tc_restart_smem(int nin, int nout) {
  const int Kp = (nin + kKc - 1) / kKc * kKc, N = (nout + 15) / 16 * 16;
  return (size_t)((3 * Kp * N * 2 + 1023) & ~1023) + 2 * kStage + 64;
}

// Host image of the three bf16 splits of Q (nin x nout, column-major FP64).
void tc_restart_bimage(int nin, int nout, const double* Q, std::vector<uint16_t>& img) {
  const int Kp = (nin + kKc - 1) / kKc * kKc, N = (nout + 15) / 16 * 16;
  img.assign((size_t)3 * Kp * N, 0);
  for (int o = 0; o < nout; ++o)
    for (int l = 0; l < nin; ++l) {
      double rem = Q[l + (size_t)o * nin];
      for (int s = 0; s < 3; ++s) {
        const uint16_t h = host_bf16((float)rem);
        rem -= host_bf16_value(h);
        img[(size_t)s * Kp * N + canon_off(o, l, N) / 2] = h;
      }
    }
}

// ---- double-float basis ----

static int df_kp(int nin) { return (nin + 15) / 16 * 16; }
static int df_n(int nout) { return (nout + 15) / 16 * 16; }

size_t tc_restart_df_smem(int nin, int nout) {
  const size_t b = (size_t)kDfDigits * df_kp(nin) * df_n(nout) * 2;
  return ((b + 1023) & ~(size_t)1023) + 2 * kDfStage + 64 + (size_t)df_kp(nin) * sizeof(int);
}

bool tc_restart_df_supported(int nin, int nout) {
  return nin >= 1 && nin <= 192 && nout >= 1 && nout <= 64 && tc_restart_df_smem(nin, nout) <= kTcDfSmemMax;
}

// Digit image of Q (nin x nout, column-major FP64) and the column exponents:
// |Q[:, o]| < 2^(f_o - 1), W = round(Q 2^(48 - f_o)) = sum_t c_t 2^(42 - 7t).
void tc_restart_df_bimage(int nin, int nout, const double* Q, std::vector<uint16_t>& img, std::vector<int>& fexp) {
  const int Kp = df_kp(nin), N = df_n(nout);
  img.assign((size_t)kDfDigits * Kp * N, 0);
  fexp.assign(N, 0);
  for (int o = 0; o < nout; ++o) {
    double mx = 0.0;
    for (int l = 0; l < nin; ++l) mx = std::max(mx, std::fabs(Q[l + (size_t)o * nin]));
    int E2 = 0;
    if (mx > 0.0) std::frexp(mx, &E2);          // mx < 2^E2
    const int f = E2 + 1;
    fexp[o] = f;
    for (int l = 0; l < nin; ++l) {
      const int64_t W = std::llround(std::ldexp(Q[l + (size_t)o * nin], 48 - f));
      for (int t = 0; t < kDfDigits; ++t) {
        const int dgt = t == 0 ? (int)(W >> 42) : (int)((W >> (42 - 7 * t)) & 127);
        img[(size_t)t * Kp * N + canon_off(o, l, N) / 2] = host_bf16((float)dgt);
      }
    }
  }
}

void launch_tc_restart_df(int64_t n, const float2* in, float2* out, int64_t ldu, int nin, int nout, const void* bimg,
                          const int* fexp, const int* pexp, int* rexp, const float2* mvsrc, float2* mvdst, int* flag,
                          cudaStream_t st) {
  const int Kp = df_kp(nin), N = df_n(nout);
  int tcols = 32;
  while (tcols < kDfGroups * N) tcols *= 2;
  const int64_t ntiles = (n + kM - 1) / kM;
  const size_t sm = tc_restart_df_smem(nin, nout);
  int sms = 152, dev = 0, per_sm = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_restart_df, kDfAllThreads, sm) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  per_sm = std::min(per_sm, 512 / tcols);          // tensor memory columns per SM
  const int ge = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  k_row_exp<<<std::max(ge, 1), 256, 0, st>>>(n, in, ldu, nin, pexp, rexp);
  const int g = (int)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
  k_tc_restart_df<<<g, kDfAllThreads, sm, st>>>(n, in, out, ldu, nin, Kp, N, nout, static_cast<const uint4*>(bimg),
                                             fexp, pexp, rexp, mvsrc, mvdst, tcols, flag);
}

static cudaError_t configure_tc_kernels_once() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_restart_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_restart_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcDfSmemMax);
  return e;
}

cudaError_t configure_tc_kernels() { return once_per_device(kCfgTc, configure_tc_kernels_once); }

void launch_tc_restart_f32(int64_t n, const float* in, float* out, int64_t ldu, int nin, int nout, const void* bimg,
                           const float* mvsrc, float* mvdst, int* flag, cudaStream_t st) {
  const int Kp = (nin + kKc - 1) / kKc * kKc, N = (nout + 15) / 16 * 16;
  const int64_t ntiles = (n + kM - 1) / kM;
  const size_t sm = tc_restart_smem(nin, nout);
  int per_sm = 1, sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_restart_f32, kThreads, sm) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  per_sm = std::min(per_sm, 512 / kTmemCols);   // tensor memory columns per SM
  const int g = (int)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
  k_tc_restart_f32<<<g, kThreads, sm, st>>>(n, in, out, ldu, nin, Kp, N, nout,
                                                                      static_cast<const uint4*>(bimg), mvsrc, mvdst,
                                                                      flag);
}

}  // namespace rks
