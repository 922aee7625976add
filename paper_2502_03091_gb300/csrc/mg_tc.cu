// mg_tc.cu -- tensor-core (tcgen05) contractions of the chiral truncation.
//
// The per-block SVD of the truncation (paper Sec. 3, Eq. 4: the K x m' block
// A = Psi^(alpha)(Lambda_j), K = 6|Lambda|, factored by CholeskyQR2 and the
// SVD of its small R factor) needs two kinds of dense contraction per
// block-chirality bc = 2j + alpha:
//   Gram:  G = A^dag A                     (m' x m', Hermitian)
//   GEMM:  C = A B                         (K x n; B an m' x n matrix of bc)
// Both are taken over the reals.  A row of A is stored as 2m' interleaved
// reals (re_0, im_0, re_1, ...), so A~ is K x 2m' and
//   Gram: (A~^T A~)[2i+a][2j+b] gives G[i][j] = (rr + ii) + i (ri - ir);
//   GEMM: C~ = A~ B~, with the 2m' x 2n real form of B
//         B~[2i][2j] = re b, B~[2i][2j+1] = im b, B~[2i+1][2j] = -im b,
//         B~[2i+1][2j+1] = re b,
//         and C~[r][2j], C~[r][2j+1] the real and imaginary parts of C[r][j].
// They run on the 5th-generation tensor cores: operands staged in shared
// memory in the K-major canonical layout (core matrices of 8 rows x 16 bytes,
// no swizzle), FP32 accumulators in TMEM, one thread issuing tcgen05.mma
// (M = 128, K = 16 per instruction, kind::f16) and tcgen05.commit to one
// mbarrier per staging buffer, tcgen05.ld epilogues.  The kernels are
// persistent: a CTA walks the block-chiralities bc = blockIdx.x,
// blockIdx.x + gridDim.x, ... in chunks of 128 rows of A.
//
// Two operand precisions:
//  * BF16, one product per pair of operands: about 2^-9 relative per product.
//    Used for the first Gram G1 = A^dag A, which only yields the
//    preconditioner R1 of CholeskyQR2's second pass.
//  * FP16 hi/lo split, three products: a value v of a block-chirality is
//    scaled by a power of two s (chosen per block-chirality so that
//    |s v| <= 2^14: no overflow, and the typical entry stays far above the
//    subnormal range), then split into h = fp16(s v) and l = fp16(s v - h).
//    x y is taken as hh + hl + lh; the dropped ll term is below 2^-22 |x y|,
//    so the contraction is accurate to about FP32 rounding.  The scales are
//    undone exactly in the epilogue.
//
// Every wait on an mbarrier is bounded.  A CTA whose wait gives up stops
// staging and issuing, waits (bounded) for the last matrix multiplies it
// committed, writes nothing more, frees its TMEM and sets bit 1 of the status
// word (mg_sync_status reports MG_ERR_TIMEOUT; the outputs of that call are
// then undefined).
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mg_bulk.cuh"
#include "mg_common.cuh"

namespace mg {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;                 // rows of A per staged chunk
constexpr int kTcCols = 128;                 // reals per row of A~ (2m' padded)
constexpr int kTcTile = kTcRows * kTcCols * 2;  // bytes of one 16-bit tile (32 KB)
constexpr int kTcSbo = (kTcCols / 8) * 128;  // bytes between 8-row groups of a tile (2048)
constexpr int kTcMaxSites = 1024;            // largest |Lambda| of a gathered block
constexpr int kTcMaxPolls = 1 << 20;

enum { TC_BF16 = 0, TC_FP16X3 = 1 };

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading-dimension
// byte offset (between core matrices adjacent in K), stride byte offset
// (between core matrices adjacent in M/N), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16 with FP32 accumulation, both operands
// K-major, M = 128: operand type 0 = FP16, 1 = BF16
__device__ __forceinline__ uint32_t idesc_f16(int n, int bf16) {
  const uint32_t t = bf16 ? 1u : 0u;
  return (1u << 4) | (t << 7) | (t << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t taddr, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

// waits for completion `use` (0-based) of the barrier; false after a bounded
// number of polls
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, int use) {
  const uint32_t parity = (uint32_t)(use & 1);
  for (int i = 0; i < kTcMaxPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   su32(slot)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t a, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// two 16-column loads of this thread's TMEM lane, one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t a, uint32_t b, float v[16], float w[16]) {
  uint32_t r[16], q[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
        "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]),
        "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
      : "r"(b));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = __uint_as_float(r[i]);
    w[i] = __uint_as_float(q[i]);
  }
}

__device__ __forceinline__ void sync_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void sync_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy writes to shared memory -> visible to the tensor core
__device__ __forceinline__ void fence_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// operand conversion: 8 values -> one 16-byte row of a core matrix
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t hf2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// PREC == TC_BF16: hi = bf16(v); TC_FP16X3: hi = fp16(s v), lo = fp16(s v - hi)
template <int PREC>
__device__ __forceinline__ void split8(const float v[8], float s, uint4& hi, uint4& lo) {
  if (PREC == TC_BF16) {
    hi = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
  } else {
    float x[8], r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[i] = v[i] * s;
      r[i] = x[i] - __half2float(__float2half_rn(x[i]));
    }
    hi = make_uint4(hf2(x[0], x[1]), hf2(x[2], x[3]), hf2(x[4], x[5]), hf2(x[6], x[7]));
    lo = make_uint4(hf2(r[0], r[1]), hf2(r[2], r[3]), hf2(r[4], r[5]), hf2(r[6], r[7]));
  }
}

// power of two s with s * bound <= 2^14 (1 for a zero or non-finite bound)
__device__ __forceinline__ float scale_for(float bound) {
  if (!(bound > 0.f) || !isfinite(bound)) return 1.f;
  int e;
  frexpf(bound, &e);  // bound <= 2^e
  return ldexpf(1.f, 14 - e);
}

// ---------------------------------------------------------------------------
// rows of A
// ---------------------------------------------------------------------------
struct TcRows {
  const float* src;  // psi [V][12][m'] (gather) or contiguous rows [bc][K][m'], complex
  int gather;
  int L[4], b[4], Lc[4];
  int nb, K, m, nbc;
};

// One complex Gram entry in double-float, the form the Gram's readers compute
// in: (re hi, re lo, im hi, im lo) in the 16 bytes of a complex FP64 entry.
struct dz2 {
  float re_hi, re_lo, im_hi, im_lo;
};
// (a + b) inv, (c + d) inv exactly (TwoSum; inv a power of two)
__device__ __forceinline__ dz2 dz2_of(float a, float b, float c, float d, float inv) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  const float t = __fadd_rn(c, d), dd = __fsub_rn(t, c);
  const float f = __fadd_rn(__fsub_rn(c, __fsub_rn(t, dd)), __fsub_rn(d, dd));
  return dz2{s * inv, e * inv, t * inv, f * inv};
}

// global site of local site `loc` of block `j`
__device__ __forceinline__ int tc_block_site(const TcRows& g, int j, int loc) {
  int jc[4], lc[4];
  int t = j;
  jc[0] = t % g.Lc[0]; t /= g.Lc[0];
  jc[1] = t % g.Lc[1]; t /= g.Lc[1];
  jc[2] = t % g.Lc[2]; jc[3] = t / g.Lc[2];
  t = loc;
  lc[0] = t % g.b[0]; t /= g.b[0];
  lc[1] = t % g.b[1]; t /= g.b[1];
  lc[2] = t % g.b[2]; lc[3] = t / g.b[2];
  return (jc[0] * g.b[0] + lc[0]) +
         g.L[0] * ((jc[1] * g.b[1] + lc[1]) +
                   g.L[1] * ((jc[2] * g.b[2] + lc[2]) + g.L[2] * (jc[3] * g.b[3] + lc[3])));
}

// per-CTA table of the float offset of each site's chirality-0 rows (gather
// mode), filled for block j; row r of chirality alpha starts at
// table[r / 6] + (6 alpha + r % 6) * 2m'
__device__ void fill_site_table(const TcRows& g, int j, long* table) {
  for (int loc = threadIdx.x; loc < g.nb; loc += blockDim.x)
    table[loc] = (long)tc_block_site(g, j, loc) * 12 * 2 * g.m;
}

__device__ __forceinline__ const float* row_ptr(const TcRows& g, const long* table, int bc,
                                                int r) {
  if (g.gather) return g.src + table[r / 6] + (long)(6 * (bc & 1) + r % 6) * 2 * g.m;
  return g.src + ((long)bc * g.K + r) * 2 * g.m;
}

// Gram staging: chunk c of bc into the transposed K-major tiles (M = column of
// A~, K = row): element (column q, row r) at (q>>3)*2048 + (r>>3)*128 +
// (q&7)*16 + (r&7)*2.  Thread t covers the columns 2(t&63), 2(t&63)+1 and the
// row groups (t>>6) + 4p; a warp reads 256 contiguous bytes of a row per load.
template <int PREC>
__device__ void stage_gram(const TcRows& g, const long* table, int bc, int c, float s,
                           unsigned char* hi, unsigned char* lo) {
  const int cp = threadIdx.x & 63, q0 = 2 * cp;
  const int nreal = 2 * g.m;
#pragma unroll 1
  for (int p2 = 0; p2 < 4; p2 += 2) {
    // two row groups' loads in flight at once (16 x 8 bytes)
    float2 x[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = c * kTcRows + ((threadIdx.x >> 6) + 4 * (p2 + h)) * 8 + i;
        x[h][i] = (r < g.K && q0 < nreal)
                      ? __ldg(reinterpret_cast<const float2*>(row_ptr(g, table, bc, r) + q0))
                      : make_float2(0.f, 0.f);
      }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int rg = (threadIdx.x >> 6) + 4 * (p2 + h);
    float v0[8], v1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      v0[i] = x[h][i].x;
      v1[i] = x[h][i].y;
    }
    uint4 h0, l0, h1, l1;
    split8<PREC>(v0, s, h0, l0);
    split8<PREC>(v1, s, h1, l1);
    // the bank group of a 16-byte store is q & 7: lanes 4..7 of each 8-lane
    // phase store their second column first, so a phase covers all 8 groups
    const uint32_t o0 = (q0 >> 3) * kTcSbo + rg * 128 + (q0 & 7) * 16;
    if ((threadIdx.x >> 2) & 1) {
      *reinterpret_cast<uint4*>(hi + o0 + 16) = h1;
      *reinterpret_cast<uint4*>(hi + o0) = h0;
      if (PREC == TC_FP16X3) {
        *reinterpret_cast<uint4*>(lo + o0 + 16) = l1;
        *reinterpret_cast<uint4*>(lo + o0) = l0;
      }
    } else {
      *reinterpret_cast<uint4*>(hi + o0) = h0;
      *reinterpret_cast<uint4*>(hi + o0 + 16) = h1;
      if (PREC == TC_FP16X3) {
        *reinterpret_cast<uint4*>(lo + o0) = l0;
        *reinterpret_cast<uint4*>(lo + o0 + 16) = l1;
      }
    }
  }
  }
}

// GEMM staging: chunk c of bc into K-major tiles (M = row, K = real column):
// element (row r, column q) at (r>>3)*2048 + (q>>3)*128 + (r&7)*16 + (q&7)*2.
// Thread t covers row t&127 and the column groups (t>>7) + 2p.  The loads
// (16 x 16 bytes per thread) are issued one chunk ahead into registers, so
// they arrive while the previous chunk's MMAs and epilogue run.
__device__ __forceinline__ void load_gemm_rows(const TcRows& g, const long* table, int bc, int c,
                                               float4 ld[16]) {
  const int rl = threadIdx.x & 127;
  const int r = c * kTcRows + rl;
  const int nreal = 2 * g.m;
  const float* rp = r < g.K ? row_ptr(g, table, bc, r) : nullptr;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int cg = (threadIdx.x >> 7) + 2 * p;
    const bool ok = rp && 8 * cg < nreal;
    ld[2 * p] = ok ? __ldg(reinterpret_cast<const float4*>(rp + 8 * cg)) : make_float4(0.f, 0.f, 0.f, 0.f);
    ld[2 * p + 1] =
        ok ? __ldg(reinterpret_cast<const float4*>(rp + 8 * cg + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}
__device__ __forceinline__ void store_gemm_rows(const float4 ld[16], float s, unsigned char* hi,
                                                unsigned char* lo) {
  const int rl = threadIdx.x & 127;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int cg = (threadIdx.x >> 7) + 2 * p;
    const float4 a = ld[2 * p], b = ld[2 * p + 1];
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint4 h, l;
    split8<TC_FP16X3>(v, s, h, l);
    const uint32_t o = (rl >> 3) * kTcSbo + cg * 128 + (rl & 7) * 16;
    *reinterpret_cast<uint4*>(hi + o) = h;
    *reinterpret_cast<uint4*>(lo + o) = l;
  }
}

// block-wide maximum of a non-negative float (all threads get it)
__device__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, red[i]);
  return r;
}

// ---------------------------------------------------------------------------
// Gram kernel: G[bc] = A^dag A (FP64 output [bc][m'][m']).
//
// The tensor core's FP32 accumulation is not round-to-nearest: on a long
// chain of accumulating MMAs (3072 rows x 3 products here) it drifts by
// about 1e-5 relative, systematically.  So the FP16X3 form keeps every TMEM
// accumulation short: per chunk of 128 rows, D1 = sum of the hi*hi products
// (8 MMAs) and D2 = sum of the hi*lo + lo*hi products (16 MMAs, 2^-11 smaller)
// start from zero, and the chunk sums D1 + D2 are added on the CUDA cores
// (round to nearest) in the registers of the epilogue warps: thread (warp w
// < 4, lane) owns row 32w + lane of the 128 x 128 result.  TMEM holds two
// slots (D1, D2) so the epilogue of chunk c-1 overlaps the MMAs of chunk c.
// The BF16 form (the preconditioner Gram) accumulates all chunks in TMEM.
// bound (FP16X3 only): per-bc bound on |entries of A| for the scale.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(kTcThreads, PREC == TC_BF16 ? 3 : 1)
    tc_gram_kernel(TcRows g, const float* bound,
                                                                double2* __restrict__ G,
                                                                int* __restrict__ status) {
  constexpr bool X3 = PREC == TC_FP16X3;
  constexpr int NP = X3 ? 2 : 1;
  constexpr int TCOLS = X3 ? 4 * kTcCols : kTcCols;  // (D1, D2) x 2 slots, or one D
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* tiles = tc_smem;                                      // [2][NP][kTcTile]
  long* table = reinterpret_cast<long*>(tc_smem + 2 * NP * kTcTile);  // [kTcMaxSites]
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) tmem_alloc(&tmem_base, TCOLS);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  sync_before();
  __syncthreads();
  sync_after();
  const uint32_t taddr = tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t idesc = idesc_f16(kTcCols, PREC == TC_BF16);
  const int nchunk = (g.K + kTcRows - 1) / kTcRows;
  const int m = g.m;
  int gidx = 0;  // chunks this CTA has committed
  int last_j = -1;
  float acc[X3 ? kTcCols : 1];  // FP16X3: this thread's row of the sum of chunk results

  // FP16X3: add the chunk in TMEM slot d to acc (warps 0-3)
  auto add_chunk = [&](int d) {
    if (!X3 || warp >= 4) return;
    sync_after();
#pragma unroll
    for (int cb = 0; cb < kTcCols / 16; ++cb) {
      float v1[16], v2[16];
      tmem_ld16(taddr + lane_base + d * 2 * kTcCols + cb * 16, v1);
      tmem_ld16(taddr + lane_base + d * 2 * kTcCols + kTcCols + cb * 16, v2);
#pragma unroll
      for (int t = 0; t < 16; ++t) acc[cb * 16 + t] += v1[t] + v2[t];
    }
  };

  for (int bc = blockIdx.x; bc < g.nbc && !s_abort; bc += gridDim.x) {
    if (g.gather && (bc >> 1) != last_j) {
      last_j = bc >> 1;
      fill_site_table(g, last_j, table);
      __syncthreads();
    }
    const float s = X3 ? scale_for(bound ? bound[bc] : 1.f) : 1.f;
    if (X3) {
#pragma unroll
      for (int i = 0; i < kTcCols; ++i) acc[i] = 0.f;
    }
    for (int c = 0; c < nchunk; ++c, ++gidx) {
      const int b = gidx & 1;
      unsigned char* hi = tiles + b * NP * kTcTile;
      unsigned char* lo = hi + kTcTile;  // (FP16X3 only)
      // the MMAs that read this buffer (and TMEM slot) two chunks ago are done
      if (gidx >= 2 && !bar_wait(&bar[b], (gidx - 2) >> 1)) s_abort = 1;
      __syncthreads();
      if (s_abort) break;
      stage_gram<PREC>(g, table, bc, c, s, hi, lo);
      fence_async();
      sync_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        sync_after();
        const uint32_t d1 = taddr + (X3 ? b * 2 * kTcCols : 0), d2 = d1 + kTcCols;
#pragma unroll 1
        for (int k = 0; k < kTcRows / 16; ++k) {
          const uint64_t dh = smem_desc(su32(hi) + k * 256, 128, kTcSbo);
          if (X3) {
            const uint64_t dl = smem_desc(su32(lo) + k * 256, 128, kTcSbo);
            mma(d1, dh, dh, idesc, k > 0 ? 1u : 0u);
            mma(d2, dh, dl, idesc, k > 0 ? 1u : 0u);
            mma(d2, dl, dh, idesc, 1u);
          } else {
            mma(d1, dh, dh, idesc, (c > 0 || k > 0) ? 1u : 0u);
          }
        }
        commit(&bar[b]);
      }
      if (X3 && c > 0) {
        // chunk c-1 (committed as gidx-1) while chunk c multiplies
        if (warp < 4 && !bar_wait(&bar[(gidx - 1) & 1], (gidx - 1) >> 1)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        add_chunk((gidx - 1) & 1);
      }
      sync_before();
      __syncthreads();
    }
    if (s_abort) break;
    // the last commit covers every MMA of this bc
    if (!bar_wait(&bar[(gidx - 1) & 1], (gidx - 1) >> 1)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    sync_after();
    if (warp < 4) {
      // lane = row rho = 32 warp + lane; rows 2i, 2i+1 (re, im of column i of
      // A) are neighbouring lanes
      const int rho = warp * 32 + lane, i = rho >> 1;
      const float inv = 1.f / (s * s);  // a power of two: the scaling is exact
      dz2* Gb = reinterpret_cast<dz2*>(G) + (long)bc * m * m;
      if (X3) add_chunk((gidx - 1) & 1);
#pragma unroll
      for (int cb = 0; cb < kTcCols / 16; ++cb) {
        float v[16];
        if (X3) {
#pragma unroll
          for (int t = 0; t < 16; ++t) v[t] = acc[cb * 16 + t];
        } else {
          tmem_ld16(taddr + lane_base + cb * 16, v);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float re_re = v[2 * t], re_im = v[2 * t + 1];
          const float im_re = __shfl_down_sync(0xffffffffu, re_re, 1);
          const float im_im = __shfl_down_sync(0xffffffffu, re_im, 1);
          const int jj = cb * 8 + t;
          if ((lane & 1) == 0 && i < m && jj < m)
            Gb[(long)i * m + jj] = dz2_of(re_re, im_im, re_im, -im_re, inv);
        }
      }
    }
    sync_before();
    __syncthreads();
  }
  // on a timeout: let the MMAs already committed finish before TMEM is freed
  if (s_abort && threadIdx.x == 0 && gidx > 0) (void)bar_wait(&bar[(gidx - 1) & 1], (gidx - 1) >> 1);
  sync_before();
  __syncthreads();
  if (warp == 0) {
    sync_after();
    tmem_dealloc(taddr, TCOLS);
  }
  if (s_abort && threadIdx.x == 0) atomicOr(status, 2);
}

// ---------------------------------------------------------------------------
// GEMM kernel: C[bc] = A B[bc] with FP16X3 operands.  B: [bc][m'][n] complex
// (row-major); C: rows [bc][K][n] complex.  Scale of A from gdiag (the
// diagonal of a Gram of A bounds every entry: |a_ri|^2 <= G_ii), else from
// abound[bc], else 1; scale of B from its largest entry.  cmax (optional):
// per-bc largest |re| or |im| of C.  As in the Gram kernel, every TMEM
// accumulation is short: per chunk, D1 = sum over the 2m'/16 K steps of the
// hi*hi products and D2 of the hi*lo + lo*hi products, added on the CUDA
// cores in the epilogue.  (D1, D2) are double buffered in TMEM, so the
// epilogue of chunk c-1 overlaps the MMAs of chunk c.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(TcRows g, const double2* __restrict__ gdiag, const float* __restrict__ abound,
                   const float2* __restrict__ B, int n, float2* __restrict__ C,
                   float* __restrict__ cmax, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const int npad = ((2 * n + 15) / 16) * 16;
  // (D1, D2) x 2 slots of npad columns, rounded up to a power of two
  const int tcols = npad <= 16 ? 64 : (npad <= 32 ? 128 : (npad <= 64 ? 256 : 512));
  unsigned char* atiles = tc_smem;                    // [2 buffers][hi, lo][kTcTile]
  unsigned char* bhi = tc_smem + 4 * kTcTile;         // [npad / 8][2048]
  unsigned char* blo = bhi + (npad / 8) * kTcSbo;
  long* table = reinterpret_cast<long*>(blo + (npad / 8) * kTcSbo);
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ float red[kTcThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) tmem_alloc(&tmem_base, tcols);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  sync_before();
  __syncthreads();
  sync_after();
  const uint32_t taddr = tmem_base;
  const uint32_t idesc = idesc_f16(npad, 0);
  const int m = g.m, nreal = 2 * m;
  const int ksteps = (nreal + 15) / 16;
  const int nchunk = (g.K + kTcRows - 1) / kTcRows;
  int gidx = 0;
  int last_j = -1;
  float inv = 1.f;
  float cm = 0.f;  // this thread's largest |C| entry of the current bc

  // epilogue of chunk cc of bc from TMEM slot d.  Its A tiles (buffer d) are
  // free once the chunk's MMAs are done, so they stage the output: warp w
  // reads TMEM lanes 32 (w & 3) .. + 31 (rows of the chunk) and the column
  // blocks cb = w >> 2, w >> 2 + 2, ..., writes them to shared memory (row
  // stride n + 1, or for n = 64 a 64-wide row with the columns XOR-swizzled
  // by the row), then every warp writes whole rows to global memory.
  auto epilogue = [&](int bc, int cc, int d) {
    sync_after();
    float2* stg = reinterpret_cast<float2*>(atiles + 2 * d * kTcTile);
    const int ld = n < 64 ? n + 1 : 64;
    const int rl = (warp & 3) * 32 + lane, r = cc * kTcRows + rl;
#pragma unroll 1
    for (int cb = warp >> 2; cb < npad / 16; cb += 2) {
      float v[16], w[16];
      const uint32_t a = taddr + ((uint32_t)((warp & 3) * 32) << 16) + d * 2 * npad + cb * 16;
      tmem_ld16(a, v);
      tmem_ld16(a + npad, w);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int jj = cb * 8 + t;
        if (jj < n) {
          const float2 z = make_float2((v[2 * t] + w[2 * t]) * inv,
                                       (v[2 * t + 1] + w[2 * t + 1]) * inv);
          stg[rl * ld + (n < 64 ? jj : (jj ^ (rl & 31)))] = z;
          if (r < g.K) cm = fmaxf(cm, fmaxf(fabsf(z.x), fabsf(z.y)));
        }
      }
    }
    __syncthreads();
    const int rows = min(kTcRows, g.K - cc * kTcRows);
    for (int row = warp; row < rows; row += kTcThreads / 32) {
      float2* out = C + ((long)bc * g.K + cc * kTcRows + row) * n;
      for (int jj = lane; jj < n; jj += 32)
        out[jj] = stg[row * ld + (n < 64 ? jj : (jj ^ (row & 31)))];
    }
  };

  for (int bc = blockIdx.x; bc < g.nbc; bc += gridDim.x) {
    if (g.gather && (bc >> 1) != last_j) {
      last_j = bc >> 1;
      fill_site_table(g, last_j, table);
    }
    // scales of A and B
    float abnd = 1.f;
    if (gdiag) {
      // the largest diagonal entry of the Gram, one per thread and a block
      // maximum (FP32 is plenty for a power-of-two scale with 4x headroom)
      const dz2* Gb = reinterpret_cast<const dz2*>(gdiag) + (long)bc * m * m;
      const float di = (int)threadIdx.x < m ? Gb[(long)threadIdx.x * m + threadIdx.x].re_hi : 0.f;
      abnd = sqrtf(block_max(di, red));
    } else if (abound) {
      abnd = abound[bc];
    }
    const float sa = scale_for(abnd);
    const float2* Bb = B + (long)bc * m * n;
    float bm = 0.f;
    for (int i = threadIdx.x; i < m * n; i += blockDim.x) {
      const float2 z = __ldg(Bb + i);
      bm = fmaxf(bm, fmaxf(fabsf(z.x), fabsf(z.y)));
    }
    const float sb = scale_for(block_max(bm, red));
    inv = 1.f / (sa * sb);
    // B~^T tiles: row n' = 2jj + bb (output real column), K column k' = 2ii + a
    for (int idx = threadIdx.x; idx < npad * (kTcCols / 8); idx += blockDim.x) {
      const int np_ = idx % npad, kg = idx / npad;
      const int jj = np_ >> 1, bb = np_ & 1;
      float v[8];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int ii = 4 * kg + t;
        float2 z = make_float2(0.f, 0.f);
        if (ii < m && jj < n) z = __ldg(Bb + (long)ii * n + jj);
        // a = 0 (re a_ii): re b / im b;  a = 1 (im a_ii): -im b / re b
        v[2 * t] = bb ? z.y : z.x;
        v[2 * t + 1] = bb ? z.x : -z.y;
      }
      uint4 h, l;
      split8<TC_FP16X3>(v, sb, h, l);
      const uint32_t o = (np_ >> 3) * kTcSbo + kg * 128 + (np_ & 7) * 16;
      *reinterpret_cast<uint4*>(bhi + o) = h;
      *reinterpret_cast<uint4*>(blo + o) = l;
    }
    cm = 0.f;
    __syncthreads();
    float4 pre[16];  // chunk c's rows, loaded during chunk c-1
    load_gemm_rows(g, table, bc, 0, pre);
    for (int c = 0; c < nchunk; ++c, ++gidx) {
      const int b = gidx & 1;
      unsigned char* ahi = atiles + 2 * b * kTcTile;
      unsigned char* alo = ahi + kTcTile;
      // the MMAs that read this buffer (and TMEM slot) two chunks ago are done
      if (gidx >= 2 && !bar_wait(&bar[b], (gidx - 2) >> 1)) s_abort = 1;
      __syncthreads();
      if (s_abort) break;
      store_gemm_rows(pre, sa, ahi, alo);
      if (c + 1 < nchunk) load_gemm_rows(g, table, bc, c + 1, pre);
      fence_async();
      sync_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        sync_after();
        const uint32_t d1 = taddr + b * 2 * npad, d2 = d1 + npad;
#pragma unroll 1
        for (int k = 0; k < ksteps; ++k) {
          const uint64_t dah = smem_desc(su32(ahi) + k * 256, 128, kTcSbo);
          const uint64_t dal = smem_desc(su32(alo) + k * 256, 128, kTcSbo);
          const uint64_t dbh = smem_desc(su32(bhi) + k * 256, 128, kTcSbo);
          const uint64_t dbl = smem_desc(su32(blo) + k * 256, 128, kTcSbo);
          mma(d1, dah, dbh, idesc, k > 0 ? 1u : 0u);
          mma(d2, dah, dbl, idesc, k > 0 ? 1u : 0u);
          mma(d2, dal, dbh, idesc, 1u);
        }
        commit(&bar[b]);
      }
      if (c > 0) {
        // chunk c-1 (committed as gidx-1) while chunk c multiplies
        if (!bar_wait(&bar[(gidx - 1) & 1], (gidx - 1) >> 1)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        epilogue(bc, c - 1, (gidx - 1) & 1);
      }
      sync_before();
      __syncthreads();
    }
    if (s_abort) break;
    // the last chunk of this bc
    if (!bar_wait(&bar[(gidx - 1) & 1], (gidx - 1) >> 1)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    epilogue(bc, nchunk - 1, (gidx - 1) & 1);
    sync_before();
    const float bcm = block_max(cm, red);  // (synchronises)
    if (cmax && threadIdx.x == 0) cmax[bc] = bcm;
  }
  if (s_abort && threadIdx.x == 0 && gidx > 0) (void)bar_wait(&bar[(gidx - 1) & 1], (gidx - 1) >> 1);
  sync_before();
  __syncthreads();
  if (warp == 0) {
    sync_after();
    tmem_dealloc(taddr, tcols);
  }
  if (s_abort && threadIdx.x == 0) atomicOr(status, 2);
}

// ---------------------------------------------------------------------------
// Galerkin coarsening D_c = P^dag D P (paper Sec. 2, Eq. 3) on the tensor
// cores.  The spin projection of the hop gives, per site x and chirality
// columns (alpha, i) of the prolongator P(x) = diag(P_0(x), P_1(x)):
//   P(x)^dag (1 - gamma_mu) U P(y) = Pi_mu(x)^dag (1_2 x U) Pi_mu(y),
//   Pi_mu = [P_0, -B_mu P_1]                (6 x 2k: 2 spins x 3 colours),
// so every term is a depth-6 product conj(L_x)^T R_x of two 6 x 2k matrices.
// Six passes per block j (as the CUDA-core coarsen_kernel):
//   passes 0, 1 (chirality alpha): L = P_alpha(x), R = 1/2 (m0 + sum w + C_alpha(x)) P_alpha(x)
//   passes 2..5 (mu = 0..3):       L = Pi_mu(x), R = hw_mu U_mu(x) Pi_mu(x + mu)
// summed over the block's sites into S (site term and hops that stay in the
// block) or, for the sites on the block's +mu face, into Y_{+mu}; then
// X = S + sigma_3 S^dag sigma_3 and Y_{-mu}(j + mu) = sigma_3 Y_{+mu}(j)^dag sigma_3.
// Over the reals, with 8 rows per site (the 6 of L or R and two zero rows)
// and chunks of 12 sites, a chunk is D = L~^T R~ with M = 4k real columns of
// L~ (padded to 128), N = 4k padded to a multiple of 32, K = 96, operands
// FP16 hi/lo (P and L scaled by 2^14: every entry of a block-orthonormal P
// is at most 1 in modulus; R by 2^8: |R| <= 64).  Per chunk D1 (hi*hi) and
// D2 (hi*lo + lo*hi) accumulate in TMEM from zero and are added on the CUDA
// cores into registers: warp w owns TMEM lanes 32 (w & 3) .. + 31 (rows of
// D) and column half w >> 2; S and Y are kept per thread.
// ---------------------------------------------------------------------------
struct TcCoarsen {
  const float2* U;
  const float2* C;
  const float2* P;
  float2* X;
  float2* Y;
  int L[4], b[4], Lc[4];
  int nb, k, nblk;
  float hw[4];
  float diag;
};

constexpr float kCsScaleL = 16384.f;           // 2^14
constexpr float kCsScaleR = 256.f;             // 2^8

// Per-NPAD layout of the coarsening kernel's shared memory:
//  * one operand tile set: L~^T (hi, lo; M = 128) and R~^T (hi, lo; N = NPAD),
//    element (real column q, row 8s + e) at (q>>3)*SBO + s*128 + (q&7)*16 + e*2;
//  * two raw buffers, each the bulk-copied inputs of one chunk: per site the
//    prolongator rows P(x) [12][k], the neighbour's P(x + mu) [12][k] (hop
//    passes) and the links U(x) [4][9] (hop passes) or the clover C(x)
//    [2][6][6] (site passes).
template <int NPAD>
struct CsCfg {
  static constexpr int S = NPAD <= 96 ? 12 : 8;        // sites per chunk (K = 8 S)
  static constexpr int KMAX = NPAD / 4;                // largest k of this NPAD
  static constexpr int SBO = S * 128;                  // bytes between 8-row groups
  static constexpr int TILE_L = (kTcCols / 8) * SBO;   // one 16-bit L~^T tile
  static constexpr int TILE_R = (NPAD / 8) * SBO;      // one 16-bit R~^T tile
  static constexpr int TILES = 2 * TILE_L + 2 * TILE_R;
  static constexpr int PST = 12 * KMAX;                // float2 per site in the P areas
  static constexpr int EST = 72;                       // float2 per site in the U / C area
  static constexpr int RAW = S * (2 * PST + EST) * 8;  // bytes of one raw buffer
};

// Pi_mu's lower-chirality columns: row sp of -B_mu has a single non-zero
// entry -B_mu[sp][t] = g
__device__ __forceinline__ void tc_pi_entry(int mu, int sp, int& t, float2& g) {
  if (mu == 0) { t = 1 - sp; g = make_float2(0.f, 1.f); }
  else if (mu == 1) { t = 1 - sp; g = make_float2(sp == 0 ? 1.f : -1.f, 0.f); }
  else if (mu == 2) { t = sp; g = make_float2(0.f, sp == 0 ? 1.f : -1.f); }
  else { t = sp; g = make_float2(-1.f, 0.f); }
}

// site t of the pass's group: group 0 = all sites (mu < 0) or the sites off
// the +mu face, group 1 = the +mu face; returns the global site and, for
// mu >= 0, its +mu neighbour
__device__ __forceinline__ int cs_site(const TcCoarsen& a, int j, int mu, int grp, int t,
                                       int* nbr) {
  int jc[4], ext[4], off[4] = {0, 0, 0, 0};
  int u = j;
  jc[0] = u % a.Lc[0]; u /= a.Lc[0];
  jc[1] = u % a.Lc[1]; u /= a.Lc[1];
  jc[2] = u % a.Lc[2]; jc[3] = u / a.Lc[2];
  for (int d = 0; d < 4; ++d) ext[d] = a.b[d];
  if (mu >= 0) {
    if (grp == 0) ext[mu] = a.b[mu] - 1;
    else { ext[mu] = 1; off[mu] = a.b[mu] - 1; }
  }
  int xo[4];
  for (int d = 0; d < 4; ++d) {
    xo[d] = jc[d] * a.b[d] + off[d] + t % ext[d];
    t /= ext[d];
  }
  const int x = xo[0] + a.L[0] * (xo[1] + a.L[1] * (xo[2] + a.L[2] * xo[3]));
  if (mu >= 0) {
    xo[mu] = (xo[mu] + 1) % a.L[mu];
    *nbr = xo[0] + a.L[0] * (xo[1] + a.L[1] * (xo[2] + a.L[2] * xo[3]));
  }
  return x;
}

// stage a chunk from its raw buffer into the L~^T and R~^T tiles; s_site[s]
// < 0 marks a site past the end of the group (zero rows)
template <int NPAD>
__device__ void cs_stage(const TcCoarsen& a, int pass, const int* s_site, const float2* raw,
                         unsigned char* lhi, unsigned char* llo, unsigned char* rhi,
                         unsigned char* rlo) {
  using Cfg = CsCfg<NPAD>;
  const int k = a.k, n2 = 2 * k;
  const int mu = pass - 2;
  const float2* rawx = raw;                      // P(x)
  const float2* rawn = raw + Cfg::S * Cfg::PST;  // P(x + mu)
  const float2* rawe = rawn + Cfg::S * Cfg::PST; // U(x) or C(x)
  // items it = r + 256 i with r = (tid + 128) mod 256: the threads that take a
  // third item are in warps 4 and 5, not in warps 0 and 1, which fetch and issue
  for (int it = (threadIdx.x + 128) & 255; it < Cfg::S * n2; it += blockDim.x) {
    const int s = it / n2, col = it % n2;
    float2 Lv[6], Rv[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) Lv[e] = Rv[e] = make_float2(0.f, 0.f);
    const int al = col / k, i = col % k;
    if (s_site[s] >= 0) {
      const float2* Px = rawx + s * Cfg::PST;  // [2][6][k]
      if (mu < 0) {
        if (al == pass) {
#pragma unroll
          for (int e = 0; e < 6; ++e) Lv[e] = Px[(al * 6 + e) * k + i];
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            float2 r = cscale(Lv[e], 0.5f * a.diag);
            if (a.C) {
              const float2* cl = rawe + s * Cfg::EST + al * 36 + e * 6;
#pragma unroll
              for (int f = 0; f < 6; ++f) cfma(r, cscale(cl[f], 0.5f), Lv[f]);
            }
            Rv[e] = r;
          }
        }
      } else {
        const float2* Py = rawn + s * Cfg::PST;
        const float2* u = rawe + s * Cfg::EST + mu * 9;
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
          int tt;
          float2 ph;
          tc_pi_entry(mu, sp, tt, ph);
          const int o = al == 0 ? (sp * 3) * k + i : (6 + tt * 3) * k + i;
          float2 py[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float2 vx = Px[o + d * k], vy = Py[o + d * k];
            Lv[sp * 3 + d] = al == 0 ? vx : cmul(ph, vx);
            py[d] = al == 0 ? vy : cmul(ph, vy);
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < 3; ++d) cfma(acc, u[c * 3 + d], py[d]);
            Rv[sp * 3 + c] = cscale(acc, a.hw[mu]);
          }
        }
      }
    }
    float lre[8], lim[8], rre[8], rim[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      lre[e] = e < 6 ? Lv[e < 6 ? e : 0].x : 0.f;
      lim[e] = e < 6 ? Lv[e < 6 ? e : 0].y : 0.f;
      rre[e] = e < 6 ? Rv[e < 6 ? e : 0].x : 0.f;
      rim[e] = e < 6 ? Rv[e < 6 ? e : 0].y : 0.f;
    }
    uint4 lhr, llr, lhm, llm, rhr, rlr, rhm, rlm;
    const int q = 2 * col;
    const uint32_t o0 = (q >> 3) * Cfg::SBO + s * 128 + (q & 7) * 16;
    split8<TC_FP16X3>(lre, kCsScaleL, lhr, llr);
    split8<TC_FP16X3>(lim, kCsScaleL, lhm, llm);
    split8<TC_FP16X3>(rre, kCsScaleR, rhr, rlr);
    split8<TC_FP16X3>(rim, kCsScaleR, rhm, rlm);
    // the bank group of a 16-byte store is q & 7: lanes 4..7 of each 8-lane
    // phase store their imaginary column first, so a phase covers all 8 groups
    const uint32_t a0 = ((threadIdx.x >> 2) & 1) ? o0 + 16 : o0, a1 = o0 + 16 - (a0 - o0);
    const bool sw = (threadIdx.x >> 2) & 1;
    *reinterpret_cast<uint4*>(lhi + a0) = sw ? lhm : lhr;
    *reinterpret_cast<uint4*>(llo + a0) = sw ? llm : llr;
    *reinterpret_cast<uint4*>(rhi + a0) = sw ? rhm : rhr;
    *reinterpret_cast<uint4*>(rlo + a0) = sw ? rlm : rlr;
    *reinterpret_cast<uint4*>(lhi + a1) = sw ? lhr : lhm;
    *reinterpret_cast<uint4*>(llo + a1) = sw ? llr : llm;
    *reinterpret_cast<uint4*>(rhi + a1) = sw ? rhr : rhm;
    *reinterpret_cast<uint4*>(rlo + a1) = sw ? rlr : rlm;
  }
}

// The chunk sequence of a CTA: blocks j = blockIdx.x, blockIdx.x + gridDim.x,
// ...; per block the site passes 0 and 1 and, per direction mu, the sites off
// the +mu face (group 0) and on it (group 1); per group, chunks of S sites.
struct CsChunk {
  int j, pass, grp, c0, cnt;
};
__device__ __forceinline__ int cs_count(const TcCoarsen& a, int pass, int grp) {
  const int mu = pass - 2;
  return mu < 0 ? a.nb : (grp == 0 ? a.nb - a.nb / a.b[mu] : a.nb / a.b[mu]);
}
template <int S>
__device__ __forceinline__ void cs_advance(const TcCoarsen& a, CsChunk& c) {
  c.c0 += S;
  while (c.j < a.nblk && c.c0 >= c.cnt) {
    c.c0 = 0;
    if (c.pass >= 2 && c.grp == 0) {
      c.grp = 1;
    } else {
      c.grp = 0;
      if (++c.pass == 6) {
        c.pass = 0;
        c.j += gridDim.x;
      }
    }
    c.cnt = cs_count(a, c.pass, c.grp);
  }
}
__device__ __forceinline__ CsChunk cs_begin(const TcCoarsen& a) {
  return CsChunk{(int)blockIdx.x, 0, 0, 0, cs_count(a, 0, 0)};
}

// warp 0: the sites of chunk c into s_site and the chunk's bulk copies into
// the raw buffer, completing on bar (lane s handles site s)
template <int NPAD>
__device__ void cs_fetch(const TcCoarsen& a, const CsChunk& c, int* s_site, float2* raw,
                         unsigned long long* bar) {
  using Cfg = CsCfg<NPAD>;
  const int lane = threadIdx.x & 31;
  const int mu = c.pass - 2;
  int x = -1, nbr = -1;
  if (lane < Cfg::S && c.c0 + lane < c.cnt) x = cs_site(a, c.j, mu, c.grp, c.c0 + lane, &nbr);
  if (lane < Cfg::S) s_site[lane] = x;
  const uint32_t pbytes = 12u * a.k * sizeof(float2);
  const uint32_t ebytes = mu >= 0 ? 36u * sizeof(float2) : (a.C ? 72u * sizeof(float2) : 0u);
  const uint32_t per_site = pbytes + (mu >= 0 ? pbytes : 0u) + ebytes;
  const int nvalid = __popc(__ballot_sync(0xffffffffu, x >= 0));
  if (lane == 0) mbar_expect_tx(bar, (uint32_t)nvalid * per_site);
  __syncwarp();
  if (x >= 0) {
    float2* rawx = raw;
    float2* rawn = raw + Cfg::S * Cfg::PST;
    float2* rawe = rawn + Cfg::S * Cfg::PST;
    bulk_g2s(rawx + lane * Cfg::PST, a.P + (long)x * 12 * a.k, pbytes, bar);
    if (mu >= 0) {
      bulk_g2s(rawn + lane * Cfg::PST, a.P + (long)nbr * 12 * a.k, pbytes, bar);
      bulk_g2s(rawe + lane * Cfg::EST, a.U + (long)x * 36, ebytes, bar);
    } else if (a.C) {
      bulk_g2s(rawe + lane * Cfg::EST, a.C + (long)x * 72, ebytes, bar);
    }
  }
}

template <int NPAD>
__global__ void __launch_bounds__(kTcThreads, 1) tc_coarsen_kernel(TcCoarsen a,
                                                                   int* __restrict__ status) {
  using Cfg = CsCfg<NPAD>;
  constexpr int NH = NPAD / 2;                        // columns per thread
  constexpr int TCOLS = 4 * NPAD <= 256 ? 256 : 512;  // (D1, D2) x 2 slots
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* lhi = tc_smem;  // one tile set; between chunks it also holds Ms
  unsigned char* llo = lhi + Cfg::TILE_L;
  unsigned char* rhi = llo + Cfg::TILE_L;
  unsigned char* rlo = rhi + Cfg::TILE_R;
  auto raw = [&](int b) { return reinterpret_cast<float2*>(tc_smem + Cfg::TILES + b * Cfg::RAW); };
  float2* Ms = reinterpret_cast<float2*>(tc_smem);  // [2k][2k + 1]
  __shared__ __align__(8) unsigned long long mma_bar;
  __shared__ __align__(8) unsigned long long raw_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ int s_site[2][Cfg::S];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = a.k, n2 = 2 * k;
  const int half = warp >> 2;
  // zero the tiles once.  The padding (real columns >= 4k of L~ and R~) is
  // never staged; between passes Ms may leave stale values there, which only
  // reach rows and columns of the product that are never read.
  for (int i = threadIdx.x; i < Cfg::TILES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(tc_smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tmem_alloc(&tmem_base, TCOLS);
  if (threadIdx.x == 0) {
    mbar_init(&mma_bar, 1);
    mbar_init(&raw_bar[0], 1);
    mbar_init(&raw_bar[1], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  sync_before();
  __syncthreads();
  sync_after();
  const uint32_t taddr = tmem_base;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t idesc = idesc_f16(NPAD, 0);
  const float inv = 1.f / (kCsScaleL * kCsScaleR);
  float Sr[NH], Yr[NH];

  // add the chunk in TMEM slot d to Sr (to_y = 0) or Yr
  auto add_chunk = [&](int d, int to_y) {
    sync_after();
#pragma unroll
    for (int cb = 0; cb < NH / 16; ++cb) {
      float v1[16], v2[16];
      const uint32_t ad = taddr + lane_base + d * 2 * NPAD + half * NH + cb * 16;
      tmem_ld16x2(ad, ad + NPAD, v1, v2);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        if (to_y) Yr[cb * 16 + t] += v1[t] + v2[t];
        else Sr[cb * 16 + t] += v1[t] + v2[t];
      }
    }
  };
  // the complex 2k x 2k matrix of the real accumulator R (this thread's row
  // and column half) into Ms
  auto to_ms = [&](bool from_y) {
    const int rho = (warp & 3) * 32 + lane, c1 = rho >> 1;
#pragma unroll
    for (int t = 0; t < NH / 2; ++t) {
      const float re_re = from_y ? Yr[2 * t] : Sr[2 * t];
      const float re_im = from_y ? Yr[2 * t + 1] : Sr[2 * t + 1];
      const float im_re = __shfl_down_sync(0xffffffffu, re_re, 1);
      const float im_im = __shfl_down_sync(0xffffffffu, re_im, 1);
      const int c2 = (half * NH) / 2 + t;
      if ((lane & 1) == 0 && c1 < n2 && c2 < n2)
        Ms[c1 * (n2 + 1) + c2] = make_float2((re_re + im_im) * inv, (re_im - im_re) * inv);
    }
  };

  // Chunk g: its inputs arrive in raw buffer g & 1 (fetched two chunks
  // ahead by warp 0), it is staged into the one tile set once the MMAs of
  // chunk g-1 are done, multiplied into TMEM slot g & 1, and added to the
  // registers one chunk later (or at once when it ends a pass).
  CsChunk cur = cs_begin(a), pre = cur;
  int issued = 0;  // chunks whose raw buffer was fetched
  if (warp == 0) {
    for (; issued < 2 && pre.j < a.nblk; ++issued) {
      cs_fetch<NPAD>(a, pre, s_site[issued], raw(issued), &raw_bar[issued]);
      cs_advance<Cfg::S>(a, pre);
    }
  }
  int pend = -1, pend_y = 0;  // TMEM slot awaiting its addition, and its target
#pragma unroll
  for (int t = 0; t < NH; ++t) Sr[t] = Yr[t] = 0.f;
  int g = 0, committed = 0;
  for (; cur.j < a.nblk; ++g) {
    const int b = g & 1;
    const int mu = cur.pass - 2;
    bool ok = mbar_wait(&raw_bar[b], (uint32_t)((g >> 1) & 1));
    if (g >= 1) ok = bar_wait(&mma_bar, g - 1) && ok;
    if (!ok) s_abort = 1;
    __syncthreads();  // s_site[b] (written by warp 0) and s_abort visible
    if (s_abort) break;
    sync_after();
    cs_stage<NPAD>(a, cur.pass, s_site[b], raw(b), lhi, llo, rhi, rlo);
    fence_async();
    sync_before();
    __syncthreads();
    if (threadIdx.x == 32) {
      sync_after();
      const uint32_t d1 = taddr + b * 2 * NPAD, d2 = d1 + NPAD;
#pragma unroll
      for (int kk = 0; kk < Cfg::S / 2; ++kk) {
        const uint64_t dlh = smem_desc(su32(lhi) + kk * 256, 128, Cfg::SBO);
        const uint64_t dll = smem_desc(su32(llo) + kk * 256, 128, Cfg::SBO);
        const uint64_t drh = smem_desc(su32(rhi) + kk * 256, 128, Cfg::SBO);
        const uint64_t drl = smem_desc(su32(rlo) + kk * 256, 128, Cfg::SBO);
        mma(d1, dlh, drh, idesc, kk > 0 ? 1u : 0u);
        mma(d2, dlh, drl, idesc, kk > 0 ? 1u : 0u);
        mma(d2, dll, drh, idesc, 1u);
      }
      commit(&mma_bar);
    }
    committed = g + 1;
    // raw buffer b is free again: fetch chunk g + 2 into it
    if (warp == 0 && pre.j < a.nblk) {
      cs_fetch<NPAD>(a, pre, s_site[b], raw(b), &raw_bar[b]);
      cs_advance<Cfg::S>(a, pre);
      ++issued;
    }
    // chunk g-1's MMAs were waited for above
    if (pend >= 0) add_chunk(pend, pend_y);
    pend = b;
    pend_y = mu >= 0 && cur.grp == 1;
    const bool pass_end = cur.c0 + Cfg::S >= cur.cnt && (mu < 0 || cur.grp == 1);
    const int j = cur.j;
    cs_advance<Cfg::S>(a, cur);
    const bool block_end = cur.j != j;
    if (mu >= 0 && pass_end) {
      // drain, then Y_{+mu}(j) and Y_{-mu}(j + mu) = sigma_3 Y_{+mu}(j)^dag sigma_3
      if (!bar_wait(&mma_bar, g)) s_abort = 1;
      __syncthreads();
      if (s_abort) break;
      add_chunk(pend, pend_y);
      pend = -1;
      sync_before();
      to_ms(true);  // Ms overlays the tiles, which the finished MMAs no longer read
      __syncthreads();
      int jc[4];
      {
        int u = j;
        jc[0] = u % a.Lc[0]; u /= a.Lc[0];
        jc[1] = u % a.Lc[1]; u /= a.Lc[1];
        jc[2] = u % a.Lc[2]; jc[3] = u / a.Lc[2];
      }
      jc[mu] = (jc[mu] + 1) % a.Lc[mu];
      const int jn = jc[0] + a.Lc[0] * (jc[1] + a.Lc[1] * (jc[2] + a.Lc[2] * jc[3]));
      for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
        const int r = idx / n2, c = idx % n2;
        a.Y[(((long)j * 8 + mu) * n2 + r) * n2 + c] = Ms[r * (n2 + 1) + c];
        float2 v = cconj(Ms[c * (n2 + 1) + r]);
        if ((r < k) != (c < k)) v = make_float2(-v.x, -v.y);
        a.Y[(((long)jn * 8 + 4 + mu) * n2 + r) * n2 + c] = v;
      }
#pragma unroll
      for (int t = 0; t < NH; ++t) Yr[t] = 0.f;
      __syncthreads();  // Ms read before the next chunk's staging overwrites the tiles
      if (block_end) {
        // X = S + sigma_3 S^dag sigma_3
        to_ms(false);
        __syncthreads();
        for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
          const int r = idx / n2, c = idx % n2;
          float2 v = cconj(Ms[c * (n2 + 1) + r]);
          if ((r < k) != (c < k)) v = make_float2(-v.x, -v.y);
          a.X[((long)j * n2 + r) * n2 + c] = cadd(Ms[r * (n2 + 1) + c], v);
        }
#pragma unroll
        for (int t = 0; t < NH; ++t) Sr[t] = 0.f;
        __syncthreads();
      }
    }
    sync_before();
    __syncthreads();
  }
  if (s_abort) {
    // let the copies and the matrix multiplies still in flight finish before
    // the CTA's shared memory and TMEM are released
    if (threadIdx.x == 0) {
      for (int h = g; h < issued; ++h) (void)mbar_wait(&raw_bar[h & 1], (uint32_t)((h >> 1) & 1));
      if (committed > 0) (void)bar_wait(&mma_bar, committed - 1);
    }
  }
  sync_before();
  __syncthreads();
  if (warp == 0) {
    sync_after();
    tmem_dealloc(taddr, TCOLS);
  }
  if (s_abort && threadIdx.x == 0) atomicOr(status, 2);
}

template <int NPAD>
size_t cs_smem(int) {
  using Cfg = CsCfg<NPAD>;
  return (size_t)Cfg::TILES + 2 * (size_t)Cfg::RAW;
}

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 148;
  return n;
}

TcRows tc_rows(const Geom& g, const float2* src, bool gather) {
  TcRows r;
  r.src = reinterpret_cast<const float*>(src);
  r.gather = gather ? 1 : 0;
  for (int i = 0; i < 4; ++i) {
    r.L[i] = g.L[i];
    r.b[i] = g.b[i];
    r.Lc[i] = g.Lc[i];
  }
  r.nb = g.nb;
  r.K = 6 * g.nb;
  r.m = g.m;
  r.nbc = (int)(2 * g.nblk);
  return r;
}

size_t gram_smem(int prec) {
  return (size_t)2 * (prec == TC_FP16X3 ? 2 : 1) * kTcTile + sizeof(long) * kTcMaxSites;
}
size_t gemm_smem(int n) {
  const int npad = ((2 * n + 15) / 16) * 16;
  return (size_t)4 * kTcTile + (size_t)2 * (npad / 8) * kTcSbo + sizeof(long) * kTcMaxSites;
}

}  // namespace

bool tc_supported(const Geom& g) {
  return g.rps == 6 && 2 * g.m <= kTcCols && g.nb <= kTcMaxSites && 2 * g.k <= kTcCols;
}

cudaError_t launch_tc_gram(const Geom& g, const float2* A, bool gather, bool fp16x3,
                           const float* bound, double2* G, int* status, cudaStream_t s,
                           const char* name) {
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(tc_gram_kernel<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gram_smem(TC_BF16));
    cudaFuncSetAttribute(tc_gram_kernel<TC_FP16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gram_smem(TC_FP16X3));
  });
  const TcRows r = tc_rows(g, A, gather);
  // BF16: three CTAs per SM fit (shared memory; 3 x 128 TMEM columns)
  const int per_sm = fp16x3 ? 1 : 3;
  const int grid = (int)std::min<long>(r.nbc, (long)num_sms() * per_sm);
  TimedScope ts(name, s);
  if (fp16x3)
    tc_gram_kernel<TC_FP16X3><<<grid, kTcThreads, gram_smem(TC_FP16X3), s>>>(r, bound, G, status);
  else
    tc_gram_kernel<TC_BF16><<<grid, kTcThreads, gram_smem(TC_BF16), s>>>(r, bound, G, status);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const Geom& g, const float2* A, bool gather, const double2* gdiag,
                           const float* abound, const float2* B, int n, float2* C, float* cmax,
                           int* status, cudaStream_t s, const char* name) {
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)gemm_smem(kTcCols / 2));
  });
  const TcRows r = tc_rows(g, A, gather);
  const int grid = (int)std::min<long>(r.nbc, (long)num_sms());
  TimedScope ts(name, s);
  tc_gemm_kernel<<<grid, kTcThreads, gemm_smem(n), s>>>(r, gdiag, abound, B, n, C, cmax,
                                                        status);
  return cudaGetLastError();
}

bool tc_coarsen_supported(const Geom& g) { return g.rps == 6 && g.k <= 32; }

cudaError_t launch_tc_coarsen(const Geom& g, const float2* U, const float2* C, const float2* P,
                              float2* X, float2* Y, int* status, cudaStream_t s) {
  TcCoarsen a;
  a.U = U;
  a.C = C;
  a.P = P;
  a.X = X;
  a.Y = Y;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.b[i] = g.b[i];
    a.Lc[i] = g.Lc[i];
    a.hw[i] = g.hw[i];
  }
  a.nb = g.nb;
  a.k = g.k;
  a.nblk = (int)g.nblk;
  a.diag = g.diag;
  const int npad = ((4 * g.k + 31) / 32) * 32;
  const int grid = (int)std::min<long>(g.nblk, (long)num_sms());
  TimedScope ts("coarsen_tc", s);
  switch (npad) {
#define MG_CS_CASE(NP)                                                                       \
  case NP: {                                                                                 \
    static PerDeviceOnce attr_once;                                                          \
    attr_once.run([&] {                                                                      \
      cudaFuncSetAttribute(tc_coarsen_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)cs_smem<NP>(NP / 4));                                        \
    });                                                                                      \
    tc_coarsen_kernel<NP><<<grid, kTcThreads, cs_smem<NP>(g.k), s>>>(a, status);             \
    break;                                                                                   \
  }
    MG_CS_CASE(32)
    MG_CS_CASE(64)
    MG_CS_CASE(96)
    MG_CS_CASE(128)
#undef MG_CS_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mg
