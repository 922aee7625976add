// mg_tc.cu -- tensor-core (tcgen05) contractions of the mixed-precision path.
//
// First Gram of the chiral truncation (Sec. 3, Eq. 4 via CholeskyQR2):
// G1 = A^dag A for every block-chirality A (K = 6|Lambda| rows of m'
// complex numbers).  With the rows stored as 2m' interleaved reals
// (re_0, im_0, re_1, ...), A~ is a real K x 2m' matrix and
//   (A~^T A~)[2i+a][2j+b],  a, b in {re, im},
// gives G1[i][j] = (re.re + im.im) + i (re.im - im.re).  A~^T A~ is one real
// 128 x 128 x K contraction (2m' padded to 128) on the 5th-generation tensor
// cores: BF16 operands staged in shared memory in the K-major canonical
// layout (8 x 16-byte core matrices, no swizzle), FP32 accumulation in TMEM,
// one elected thread issuing tcgen05.mma (M = N = 128, K = 16 per
// instruction) and tcgen05.commit to an mbarrier per staging buffer.  Both
// MMA operands are the same shared-memory tile.
//
// BF16 rounding of A perturbs G1 by about 2^-9 |A|^2 / sqrt(K) per entry;
// CholeskyQR2's second pass (FP32 Gram of Q1 = A R1^-1) restores the
// orthonormality, so only R1 (the preconditioner of the second pass) sees it.
#include <cstdint>

#include <cuda_bf16.h>

#include "mg_common.cuh"

namespace mg {
namespace {

constexpr int kTcN = 128;                    // padded 2m' = M = N of the MMA
constexpr int kTcKC = 64;                    // rows of A per staged chunk
constexpr int kTcTile = kTcN * kTcKC * 2;    // bytes of one BF16 chunk (16 KB)
constexpr int kTcSmem = 48 * 1024;           // dynamic shared memory: caps the CTAs per
                                             // SM at 4 = 512 TMEM columns / 128
constexpr int kTcMaxPolls = 1 << 20;

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

__device__ __forceinline__ bool bar_wait(unsigned long long* bar, uint32_t parity) {
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

struct TcGeom {
  int L[4], b[4], Lc[4];
  int nb, m;
};

__device__ __forceinline__ int tc_block_site(const TcGeom& g, int j, int loc) {
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

// One CTA (8 warps) per block-chirality.  Staging: warp w converts rows
// 8w .. 8w+7 of the chunk, two rows at a time (a BF16 pair along K per
// 4-byte store); lane l covers the reals 4l .. 4l+3 of a row.
__global__ void __launch_bounds__(256) gram_tc_kernel(const float* __restrict__ psi,
                                                      double2* __restrict__ G, TcGeom g,
                                                      int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bc = blockIdx.x, j = bc >> 1, al = bc & 1;
  const int m = g.m, K = 6 * g.nb, nreal = 2 * m;
  unsigned char* tile0 = tc_smem;
  unsigned char* tile1 = tc_smem + kTcTile;
  // zero both tiles: rows >= 2m' (padding) are never written again
  for (int i = tid; i < 2 * kTcTile / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(tc_smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "r"(kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_base;
  // instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const int nchunk = (K + kTcKC - 1) / kTcKC;
  bool ok = true;
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1;
    unsigned char* tile = b ? tile1 : tile0;
    // the MMAs that read this buffer two chunks ago must have completed
    if (c >= 2 && !bar_wait(&bar[b], ((c - 2) >> 1) & 1)) ok = false;
    for (int rr = 0; rr < 8; rr += 2) {
      const int kk = warp * 8 + rr;
      const int r0 = c * kTcKC + kk;
      float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
      if (4 * lane < nreal) {
        if (r0 < K) {
          const int x = tc_block_site(g, j, r0 / 6);
          v0 = __ldg(reinterpret_cast<const float4*>(psi + ((long)x * 12 + 6 * al + r0 % 6) * nreal) +
                     lane);
        }
        if (r0 + 1 < K) {
          const int x = tc_block_site(g, j, (r0 + 1) / 6);
          v1 = __ldg(reinterpret_cast<const float4*>(
                         psi + ((long)x * 12 + 6 * al + (r0 + 1) % 6) * nreal) +
                     lane);
        }
        const float a0[4] = {v0.x, v0.y, v0.z, v0.w}, a1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int mr = 4 * lane + q;  // real column of A~ = row of the K-major operand
          const uint32_t off = (mr >> 3) * 1024 + (kk >> 3) * 128 + (mr & 7) * 16 + (kk & 7) * 2;
          *reinterpret_cast<__nv_bfloat162*>(tile + off) = __floats2bfloat162_rn(a0[q], a1[q]);
        }
      }
    }
    // generic-proxy writes -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int s = 0; s < kTcKC / 16; ++s) {
        // K step s: core-matrix columns 2s, 2s+1 (LBO 128 B), row groups every 1024 B
        const uint64_t d = smem_desc(su32(tile) + s * 256, 128, 1024);
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
            "l"(d), "l"(d), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&bar[b]))
          : "memory");
    }
  }
  // the last two chunks' MMAs (every earlier one was waited for in the loop)
  if (!bar_wait(&bar[(nchunk - 1) & 1], ((nchunk - 1) >> 1) & 1)) ok = false;
  if (nchunk >= 2 && !bar_wait(&bar[(nchunk - 2) & 1], ((nchunk - 2) >> 1) & 1)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  // epilogue: warp w (< 4) holds D rows 32w + lane; rows 2i and 2i+1 (real and
  // imaginary parts of column i of A) sit in neighbouring lanes
  if (warp < 4) {
    const int rho = warp * 32 + lane;
    const int i = rho >> 1;
    double2* Gb = G + (long)bc * m * m;
    for (int cb = 0; cb < kTcN / 32; ++cb) {
      uint32_t r[32];
      const uint32_t a = taddr + ((uint32_t)(warp * 32) << 16) + cb * 32;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(a));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        // D[2i][2jj], D[2i][2jj+1] here; D[2i+1][2jj], D[2i+1][2jj+1] in lane + 1
        const float re_re = __uint_as_float(r[2 * t]), re_im = __uint_as_float(r[2 * t + 1]);
        const float im_re = __shfl_down_sync(0xffffffffu, re_re, 1);
        const float im_im = __shfl_down_sync(0xffffffffu, re_im, 1);
        const int jj = cb * 16 + t;
        if ((lane & 1) == 0 && i < m && jj < m)
          Gb[(long)i * m + jj] =
              make_double2((double)re_re + (double)im_im, (double)re_im - (double)im_re);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcN)
                 : "memory");
  }
  if (!ok && tid == 0) atomicOr(status, 2);
}

}  // namespace

bool gram_tc_supported(const Geom& g) { return 2 * g.m <= kTcN; }

cudaError_t launch_gram_tc(const Geom& g, const float2* psi, double2* G, int* status,
                           cudaStream_t s) {
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  });
  TcGeom tg;
  for (int i = 0; i < 4; ++i) {
    tg.L[i] = g.L[i];
    tg.b[i] = g.b[i];
    tg.Lc[i] = g.Lc[i];
  }
  tg.nb = g.nb;
  tg.m = g.m;
  TimedScope ts("trunc_gram_tc", s);
  gram_tc_kernel<<<(int)(2 * g.nblk), 256, kTcSmem, s>>>(reinterpret_cast<const float*>(psi), G,
                                                         tg, status);
  return cudaGetLastError();
}

}  // namespace mg
