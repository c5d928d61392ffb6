// Dense complex64 product Y = A B (n x n, row-major) on the 5th-generation tensor cores, for
// the adjoint of the table build: Y = Gbar G, whose diagonal against G gives dT/dV_k =
// 2 Re (G Gbar G)_kk (the paper does not differentiate its estimator; the derivation is in
// k_backward.cu).
//
// The complex product is one real product with M = n, K' = 2n, N' = 2n:
//   A'[i][2k] = Re A[i][k], A'[i][2k+1] = Im A[i][k]        (A' is A's memory read as floats)
//   B'[2k][j]     = Re B[k][j], B'[2k+1][j]     = -Im B[k][j]   (column j: Re Y[i][j])
//   B'[2k][n+j]   = Im B[k][j], B'[2k+1][n+j]   =  Re B[k][j]   (column n + j: Im Y[i][j])
// in 3xTF32: each operand is split into its TF32 rounding (hi) and the exact FP32 remainder
// (lo), and D = A'_lo B'_hi + A'_hi B'_lo + A'_hi B'_hi accumulates in FP32 (the dropped
// lo x lo term is below FP32 rounding).
//
// One CTA (4 warps) computes a block of 128 rows x 64 complex columns: D in TMEM (128 lanes x
// 128 FP32 columns: Re Y then Im Y), k in stages of 16 complex (K' = 32).  Per stage the
// threads load the A tile (coalesced: a warp reads two rows' segments) and a quarter of the B
// column segments each into registers, wait until the MMAs of the stage two back have
// released the buffers, pass the A tile through shared memory so that thread t holds row t
// (TMEM lane t), write the split operands (A to TMEM with tcgen05.st, B to shared memory in
// the K-major core-matrix layout), and one thread issues the 12 MMAs (3 splits x 4 K-steps of
// 8) and commits them to the stage's mbarrier.  Loads of stage t overlap the MMAs of stage
// t - 1.  Every mbarrier wait is bounded; a timeout sets ERR_TIMEOUT.
#include <cuda_runtime.h>

#include "negf_internal.cuh"
#include "tcgen05.cuh"

namespace negf {
namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kTileM = 128;                 // rows of Y per CTA (TMEM lanes)
constexpr int kTileC = 64;                  // complex columns of Y per CTA: N' = 128
constexpr int kTileK = 16;                  // complex k per stage: K' = 32 TF32
constexpr uint32_t kTmemCols = 256;         // D: 0..127; stage s: A hi at 128 + 64 s, lo + 32
constexpr uint32_t kColD = 0, kColA = 128;
constexpr uint32_t kLBO = 128, kSBO = 1024; // 8 core matrices (K' = 32) per 8-row group
constexpr size_t kBSplit = (size_t)2 * kTileC * 32 * 4;   // one B split of one stage: 16 KB
constexpr int kAPitch = kTileK + 1;         // A tile staging [row][k], padded
constexpr size_t kABytes = (size_t)kTileM * kAPitch * sizeof(cf);
// two stages x (hi, lo) of B, the A staging, two mbarriers and the TMEM address
constexpr size_t kSmemUsed = 4 * kBSplit + kABytes + 64;
// the output staging of the epilogue reuses the operand buffers
static_assert((size_t)kTileM * (kTileC + 1) * sizeof(cf) <= 4 * kBSplit + kABytes,
              "epilogue staging must fit the operand buffers");
// at least 100 KB, so that at most two CTAs (2 x 256 TMEM columns) share an SM
constexpr size_t kSmem = kSmemUsed > 100 * 1024 ? kSmemUsed : 100 * 1024;
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ void split_tf32(float x, uint32_t& h, uint32_t& l) {
  h = to_tf32(x);
  l = __float_as_uint(x - __uint_as_float(h));
}

// byte offset of B'^T row nn, K' chunk q (4 TF32) in the core-matrix layout
__device__ __forceinline__ uint32_t b_off(int nn, int q) {
  return (uint32_t)(nn >> 3) * kSBO + (uint32_t)q * kLBO + (uint32_t)(nn & 7) * 16u;
}

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity) {
  bool got = false;
  for (uint32_t it = 0; it < kWaitLimit && !got; ++it) got = mbar_try_wait(bar, parity);
  return got;
}

__global__ void __launch_bounds__(kThreads, 1) cgemm_tc_kernel(const cf* __restrict__ A,
                                                               const cf* __restrict__ B,
                                                               cf* __restrict__ Y, int n,
                                                               int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  cf* sA = reinterpret_cast<cf*>(smem + 4 * kBSplit);                 // A tile [row][k]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 4 * kBSplit + kABytes);   // per stage
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tmem_alloc(s_tmem, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *s_tmem;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);   // this warp's lane quarter

  const int i0 = blockIdx.y * kTileM, c0 = blockIdx.x * kTileC;
  const int bc = tid & (kTileC - 1);           // B column c0 + bc, k half tid >> 6
  const int col = c0 + bc;
  const int kh = (tid >> 6) * (kTileK / 2);
  // instruction descriptor: D F32, A and B TF32, K-major both, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) |
                         ((128u >> 4) << 24);
  const int nk = (n + kTileK - 1) / kTileK;
  bool timeout = false;
  for (int t = 0; t < nk; ++t) {
    const int st = t & 1;
    const int k0 = t * kTileK;
    // this stage's operands into registers (zero outside the matrix): A element e = tid +
    // 128 q is (row e / 16, k e % 16) of the tile
    cf av[kTileK], bv[kTileK / 2];
#pragma unroll
    for (int q = 0; q < kTileK; ++q) {
      const int e = tid + kThreads * q;
      const int r = i0 + e / kTileK, k = k0 + e % kTileK;
      av[q] = (r < n && k < n) ? A[(uint64_t)r * n + k] : cf{0.f, 0.f};
    }
#pragma unroll
    for (int q = 0; q < kTileK / 2; ++q) {
      const int k = k0 + kh + q;
      bv[q] = (col < n && k < n) ? B[(uint64_t)k * n + col] : cf{0.f, 0.f};
    }
    // the buffers of this stage were last read by the MMAs of stage t - 2
    if (t >= 2 && !wait_bounded(&mbar[st], (uint32_t)((t - 2) >> 1) & 1u)) timeout = true;
    if (__syncthreads_or(timeout)) {
      timeout = true;
      break;
    }
    tc_fence_after();
#pragma unroll
    for (int q = 0; q < kTileK; ++q) {
      const int e = tid + kThreads * q;
      sA[(e / kTileK) * kAPitch + e % kTileK] = av[q];
    }
    __syncthreads();
    // A': lane tid (row i0 + tid), TMEM columns 2q (Re) and 2q + 1 (Im), hi and lo
    {
      uint32_t ah[32], al[32];
#pragma unroll
      for (int q = 0; q < kTileK; ++q) {
        const cf v = sA[tid * kAPitch + q];
        split_tf32(v.x, ah[2 * q], al[2 * q]);
        split_tf32(v.y, ah[2 * q + 1], al[2 * q + 1]);
      }
      tmem_st32(tlane + kColA + 64u * st, ah);
      tmem_st32(tlane + kColA + 64u * st + 32u, al);
    }
    // B'^T rows bc (Re outputs) and kTileC + bc (Im outputs), K' chunks of this k half
    unsigned char* bh = smem + (size_t)st * 2 * kBSplit;
    unsigned char* bl = bh + kBSplit;
#pragma unroll
    for (int m = 0; m < kTileK / 4; ++m) {
      const cf v0 = bv[2 * m], v1 = bv[2 * m + 1];
      const int q = (kh + 2 * m) >> 1;         // chunk of K' = 2 (kh + 2m)
      uint4 h, l;
      split_tf32(v0.x, h.x, l.x);
      split_tf32(-v0.y, h.y, l.y);
      split_tf32(v1.x, h.z, l.z);
      split_tf32(-v1.y, h.w, l.w);
      *reinterpret_cast<uint4*>(bh + b_off(bc, q)) = h;
      *reinterpret_cast<uint4*>(bl + b_off(bc, q)) = l;
      split_tf32(v0.y, h.x, l.x);
      split_tf32(v0.x, h.y, l.y);
      split_tf32(v1.y, h.z, l.z);
      split_tf32(v1.x, h.w, l.w);
      *reinterpret_cast<uint4*>(bh + b_off(kTileC + bc, q)) = h;
      *reinterpret_cast<uint4*>(bl + b_off(kTileC + bc, q)) = l;
    }
    tmem_st_wait();
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint64_t dh = smem_desc(smem_u32(bh), kLBO, kSBO);
      const uint64_t dl = smem_desc(smem_u32(bl), kLBO, kSBO);
      const uint32_t a_hi = tbase + kColA + 64u * st, a_lo = a_hi + 32u;
#pragma unroll
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t acol = pass == 0 ? a_lo : a_hi;
        const uint64_t bd = pass == 1 ? dl : dh;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint32_t acc = (t | pass | s) ? 1u : 0u;
          mma_tf32_ts(tbase + kColD, acol + (uint32_t)s * 8u,
                      bd + (uint64_t)((s * 2 * kLBO) >> 4), idesc, acc);
        }
      }
      mma_commit(&mbar[st]);
    }
  }
  // the last stage's commit covers every MMA issued before it
  if (!timeout && nk > 0) {
    const int tl = nk - 1;
    if (!wait_bounded(&mbar[tl & 1], (uint32_t)(tl >> 1) & 1u)) timeout = true;
  }
  timeout = __syncthreads_or(timeout);
  tc_fence_after();
  if (!timeout) {
    // D -> shared memory (thread t: row t; the TMEM loads are warp-collective), then out by
    // coalesced rows
    cf* stg = reinterpret_cast<cf*>(smem);                   // [row][col], pitch kTileC + 1
#pragma unroll
    for (int h = 0; h < kTileC / 32; ++h) {
      uint32_t re[32], im[32];
      tmem_ld32(tlane + kColD + 32u * h, re);
      tmem_ld32(tlane + kColD + kTileC + 32u * h, im);
      tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 32; ++e)
        stg[tid * (kTileC + 1) + 32 * h + e] = cf{__uint_as_float(re[e]), __uint_as_float(im[e])};
    }
    __syncthreads();
    for (int e = tid; e < kTileM * kTileC; e += kThreads) {
      const int r = e / kTileC, c = e % kTileC;
      if (i0 + r < n && c0 + c < n) Y[(uint64_t)(i0 + r) * n + c0 + c] = stg[r * (kTileC + 1) + c];
    }
  }
  if (timeout) {
    if (tid == 0) atomicOr(err, ERR_TIMEOUT);
    // products may still be in flight: give the last commit one more bounded wait
    if (nk > 0) wait_bounded(&mbar[(nk - 1) & 1], (uint32_t)((nk - 1) >> 1) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, kTmemCols);
}

}  // namespace

cudaError_t launch_cgemm_tc(const cf* A, const cf* B, cf* Y, int n, int32_t* err,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(cgemm_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((n + kTileC - 1) / kTileC), (unsigned)((n + kTileM - 1) / kTileM));
  cgemm_tc_kernel<<<grid, kThreads, kSmem, s>>>(A, B, Y, n, err);
  return cudaGetLastError();
}

}  // namespace negf
