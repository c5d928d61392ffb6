// Block-column propagation of the RGF for W = 64 slices in FP32 on the CUDA cores, one CTA per
// pair of block columns (Sec. III.B): G_{k,m} = -t g^L_k G_{k+1,m} towards slice 0 and
// G_{k,m} = -t g^R_k G_{k-1,m} towards slice L - 1, each block emitted as the Step 6' weights
// w_{(m,b),(k,a)} = eta_{k,a} |G_{k,m}[a][b]|^2 of the column's W rows (Eq. draw_i_simult) and,
// at the boundary slices, the lead weights <psi_b|Gamma|psi_b> = sum_nu Gamma_nu
// |(Phi^T G_{k,m})_{nu b}|^2.  Same weights as chain_kernel (one warp per column), computed
// by 512 threads with the two columns side by side: X_k [64][128] = (-t g_k) [64][64] X_{k+1}
// in shared memory, FP32 fused multiply-adds, each thread a 4 x 4 block of outputs (four warps
// per scheduler to hide the shared-memory and dependency latencies).
//
// W = 64 uses the symmetry G = G^T (H real symmetric, every self-energy a complex symmetric
// matrix), which halves the products: only the chains towards slice 0 run (and the one of the
// lead-L injection column towards slice L - 1).  A block G_{k,m} (k < m) of site column m gives
// besides the rows (m, b) the rows (k, a) of slice k towards slice m:
// w_{(k,a),(m,b)} = eta_{m,b} |G_{(m,b),(k,a)}|^2 = eta_{m,b} |G_{k,m}[a][b]|^2, and the block
// (G Phi_R)_k of the lead-R injection column gives the lead-R weights of the rows of slice k:
// <psi|Gamma_R|psi> = sum_nu Gamma_nu |(Phi_R^T G_{L-1,k})_{nu a}|^2 = sum_nu Gamma_nu
// |(G Phi_R)_k[a][nu]|^2.  Every weight is written by exactly one job.
//
// Two-level tables of W = 64 (l2_fused): each step's blocks are the 64 weights of a (row,
// slice) pair, exactly what a level-2 block of a two-level table draws from, so the kernel
// writes the block (level2.cuh: the inverse-CDF thresholds of the slice, the same arithmetic
// as the level-2 pass) and the slice's level-1 weight instead of the weights: the rows x K
// weights are never stored or read back.
#include <cuda_runtime.h>
#include <math.h>

#include "level2.cuh"
#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr int kW = 64;
constexpr int kN = 2 * kW;                    // two columns side by side
constexpr int kThreads = 512;
constexpr int kWtPitch = kW + 1;              // padded row of the weight staging
// Gs, the X ping-pong pair, the weights staging and (level-2 blocks built in the kernel) the
// staging of the transposed rows' weights
constexpr size_t kSmem = sizeof(cf) * (kW * kW + 2 * kW * kN) + 2 * sizeof(float) * kN * kWtPitch;
constexpr int kB2 = 8 + kW;                   // level-2 block of a 64-site slice: guide + octets

// eta |G|^2 with every rounding explicit, so that the weight of a (row, site) pair has the same
// bits wherever it is formed (stored weights, or a level-2 block built in the kernel)
__device__ __forceinline__ float wsq(float e, cf v) {
  return __fmul_rn(e, __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
}

__global__ void __launch_bounds__(kThreads, 1) chain_cta_kernel(
    const TaskDesc* __restrict__ tasks, const TcJob* __restrict__ jobs,
    const float* __restrict__ eta32, const float* __restrict__ phi32,
    const double* __restrict__ gam, const cf* __restrict__ gL, const cf* __restrict__ gR,
    const cf* __restrict__ start, float* __restrict__ weights, uint64_t* __restrict__ tab,
    int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  cf* Gs = reinterpret_cast<cf*>(smem);                    // [a][c]; also Phi at the edges
  cf* Xa = Gs + kW * kW;                                   // [c][b'] ping
  cf* Xb = Xa + kW * kN;                                   // [c][b'] pong
  float* Wt = reinterpret_cast<float*>(Xb + kW * kN);      // [b'][a] weights staging
  float* Wt2 = Wt + kN * kWtPitch;                         // fused: transposed rows [r][b]

  const int tid = threadIdx.x;
  const TcJob job = jobs[blockIdx.x];
  const TaskDesc d = tasks[job.task];
  const int L = d.L, n = d.n, K = d.K;
  const int dir = job.dir;
  auto m0_of = [&](int yy) { return yy < L ? yy : (yy == L ? 0 : L - 1); };
  const int ys[2] = {job.y0, job.y1};
  const float mt = (float)(-d.t);
  const float* eta = eta32 + d.onsite_off / 2;
  const cf* gsrc = (dir == 0 ? gL : gR) + d.g_off;
  float* wt = weights + d.wt_off;
  const bool fused = d.l2_fused != 0;
  float* l1 = weights + d.l1w_off;                         // fused: level-1 weights [rows][L+2]
  uint32_t* l2 = reinterpret_cast<uint32_t*>(tab + d.tab_off);   // fused: [rows][L][kB2]
  bool bad = false;
  auto row_of = [&](int y, int b) -> uint64_t {
    return y < L ? (uint64_t)y * kW + b : (uint64_t)n + (uint64_t)(y - L) * kW + b;
  };
  // fused: the level-2 blocks of a step, one per pair of adjacent threads (block bi = tid / 2,
  // half h = tid % 2: the block's weights wrow[0..63], the pair's `have`, row and slice), their
  // thresholds in registers (level2_fp32_pair); staged in shared memory 128 at a time (the two
  // weight stagings, free once read) and written block by block, 18 lanes per 288-byte block,
  // so that the stores stay contiguous
  uint64_t* blk_row = reinterpret_cast<uint64_t*>(Gs);     // Gs is free outside the product
  int* blk_slice = reinterpret_cast<int*>(blk_row + kN);
  auto put_blocks = [&](bool have, uint64_t row, int slice, const float* wrow) {
    const int h = tid & 1, bi = tid >> 1;
    uint32_t c[32];
    float tot = 0.f;
    const bool ok = level2_fp32_pair([&](int a) { return wrow[32 * h + a]; }, h, c, &tot);
    if (have) bad |= !ok;
    __syncthreads();                                       // every weight row has been read
    // 2 x 128 x 65 >= 128 x 76 words; pitch 76 (not 72): 16-byte stores of neighbouring
    // blocks start on different bank groups
    constexpr int kSP = kB2 + 4;
    uint32_t* stage = reinterpret_cast<uint32_t*>(Wt);
    for (int half = 0; half < 2; ++half) {
      const int b = bi & (kN - 1);
      if ((bi >> 7) == half) {
        if (h == 0) {
          blk_row[b] = have ? row : ~0ull;
          blk_slice[b] = slice;
          if (have) l1[row * (L + 2) + slice] = tot;
        }
        if (have) {
          uint32_t* dst = stage + b * kSP;
          // guide: the last threshold of octets 0..6 (octet 7's is 2^31); lane h holds octets
          // 4h .. 4h + 3
          *reinterpret_cast<uint4*>(dst + 4 * h) =
              make_uint4(c[7], c[15], c[23], h == 0 ? c[31] : kCdfOne);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            *reinterpret_cast<uint4*>(dst + 8 + 32 * h + 4 * i) =
                make_uint4(c[4 * i], c[4 * i + 1], c[4 * i + 2],
                           (h == 1 && i == 7) ? kCdfOne : c[4 * i + 3]);
        }
      }
      __syncthreads();
      for (int i = tid; i < kN * (kB2 / 4); i += kThreads) {
        const int bb = i / (kB2 / 4), q = i - bb * (kB2 / 4);
        const uint64_t r = blk_row[bb];
        if (r != ~0ull)
          *reinterpret_cast<uint4*>(l2 + (r * L + blk_slice[bb]) * kB2 + 4 * q) =
              *reinterpret_cast<const uint4*>(stage + bb * kSP + 4 * q);
      }
      __syncthreads();
    }
  };
  // start block of column slot col into X[:, col*64 .. col*64+63]
  auto load_start = [&](cf* X, int col) {
    const cf* st = start + d.start_off + (uint64_t)ys[col] * kW * kW;
    for (int i = tid; i < kW * kW; i += kThreads) {
      const int c = i / kW, b = i % kW;
      X[c * kN + col * kW + b] = st[i];
    }
  };
  // weights of slice k for the columns in `mask` from X (and lead weights at a boundary slice);
  // fused, also the level-2 blocks of the rows (k, a) towards the site columns in `tmask`
  // (their slice ys[col], weights eta_{y,b} |G_{k,y}[a][b]|^2): one block per thread, the
  // columns' rows on threads 0..127 and the transposed rows on 128..255
  auto emit = [&](const cf* X, int k, unsigned mask, unsigned tmask) {
    for (int i = tid; i < kN * kW; i += kThreads) {
      const int r = i % kN, a = i / kN;                    // r consecutive across threads
      Wt[r * kWtPitch + a] = wsq(eta[k * kW + a], X[a * kN + r]);
    }
    if (tmask) {
      for (int i = tid; i < kN * kW; i += kThreads) {
        const int r = i / kW, b = i % kW, col = r / kW;
        if (tmask & (1u << col))
          Wt2[r * kWtPitch + b] = wsq(eta[ys[col] * kW + b], X[(r % kW) * kN + col * kW + b]);
      }
    }
    __syncthreads();
    if (!fused) {
      for (int i = tid; i < kN * kW; i += kThreads) {
        const int a = i % kW, r = i / kW;                  // a consecutive: coalesced rows
        const int col = r / kW;
        if (mask & (1u << col))
          wt[row_of(ys[col], r % kW) * K + (uint64_t)k * kW + a] = Wt[r * kWtPitch + a];
      }
    } else {
      // every thread takes part (the stores go through barriers): pairs 0..127 a row of the
      // columns, 128..255 a transposed row
      const int bi = tid >> 1;
      bool have;
      uint64_t row;
      int slice;
      const float* wrow;
      if (bi < kN) {
        have = mask & (1u << (bi / kW));
        row = have ? row_of(ys[bi / kW], bi % kW) : 0;
        slice = k;
        wrow = Wt + bi * kWtPitch;
      } else {
        const int r = bi - kN, col = r / kW;
        have = tmask & (1u << col);
        row = (uint64_t)k * kW + r % kW;
        slice = have ? ys[col] : 0;
        wrow = Wt2 + r * kWtPitch;
      }
      put_blocks(have, row, slice, wrow);
    }
    if (k == 0 || k == L - 1) {
      // lead weights: Phi (FP32) staged in Gs (free outside the product)
      float* phis = reinterpret_cast<float*>(Gs);
      float* gams = phis + kW * kW;
      __syncthreads();
      for (int i = tid; i < kW * kW; i += kThreads) phis[i] = phi32[d.phi_off + i];
      for (int i = tid; i < kW; i += kThreads) gams[i] = (float)gam[d.lead_off + i];
      __syncthreads();
      const int r = tid % kN, h = tid / kN;                // four quarters of the modes
      float part = 0.f;
      for (int nu = h * 16; nu < h * 16 + 16; ++nu) {
        float zr = 0.f, zi = 0.f;
        for (int a = 0; a < kW; ++a) {
          const float p = phis[a * kW + nu];
          const cf v = X[a * kN + r];
          zr += p * v.x;
          zi += p * v.y;
        }
        part += gams[nu] * (zr * zr + zi * zi);
      }
      Wt[r * kWtPitch + h] = part;                         // staging is free again
      __syncthreads();
      if (h == 0) {
        const int col = r / kW;
        if (mask & (1u << col)) {
          const float lw = (Wt[r * kWtPitch] + Wt[r * kWtPitch + 1]) +
                           (Wt[r * kWtPitch + 2] + Wt[r * kWtPitch + 3]);
          const uint64_t row = row_of(ys[col], r % kW);
          if (fused) {
            if (k == 0) l1[row * (L + 2) + L] = lw;
            if (k == L - 1) l1[row * (L + 2) + L + 1] = lw;
          } else {
            if (k == 0) wt[row * K + n] = lw;
            if (k == L - 1) wt[row * K + n + 1] = lw;
          }
        }
      }
    }
    __syncthreads();
  };

  unsigned have = 0;
  for (int col = 0; col < 2; ++col)
    if (ys[col] >= 0) have |= 1u << col;
  // direction 0 emits every column's start slice
  if (dir == 0) {
    for (int col = 0; col < 2; ++col) {
      if (!(have & (1u << col))) continue;
      load_start(Xa, col);
      __syncthreads();
      emit(Xa, m0_of(ys[col]), 1u << col, 0u);
    }
  }
  const int m0a = m0_of(job.y0), m0b = job.y1 >= 0 ? m0_of(job.y1) : m0a;
  const int k_first = dir == 0 ? max(m0a, m0b) - 1 : min(m0a, m0b) + 1;
  const int k_end = dir == 0 ? -1 : L;
  const int kstep = dir == 0 ? -1 : 1;
  cf* Xc = Xa;
  cf* Xn = Xb;
  const int ty = tid / 32, tx = tid % 32;                  // outputs a = ty + 16i, b' = tx + 32j
  // this thread's share of the next step's g block, fetched while the current step multiplies
  constexpr int kGPer = kW * kW / kThreads;
  cf gnext[kGPer];
  auto fetch = [&](int k) {
    const cf* gk = gsrc + (uint64_t)k * kW * kW;
#pragma unroll
    for (int q = 0; q < kGPer; ++q) gnext[q] = gk[tid + q * kThreads];
  };
  if (k_first != k_end) fetch(k_first);
  for (int k = k_first; k != k_end; k += kstep) {
    unsigned active = 0;
    for (int col = 0; col < 2; ++col) {
      if (!(have & (1u << col))) continue;
      const int m0 = m0_of(ys[col]);
      if (dir == 0 ? k < m0 : k > m0) active |= 1u << col;
      if (dir == 0 ? k == m0 - 1 : k == m0 + 1) load_start(Xc, col);
    }
#pragma unroll
    for (int q = 0; q < kGPer; ++q) Gs[tid + q * kThreads] = cf{mt * gnext[q].x, mt * gnext[q].y};
    __syncthreads();
    if (k + kstep != k_end) fetch(k + kstep);
    float accr[4][4], acci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = 0.f;
#pragma unroll 4
    for (int c = 0; c < kW; ++c) {
      cf g[4], x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) g[i] = Gs[(ty + 16 * i) * kW + c];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xc[c * kN + tx + 32 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fmaf(g[i].x, x[j].x, accr[i][j]);
          accr[i][j] = fmaf(-g[i].y, x[j].y, accr[i][j]);
          acci[i][j] = fmaf(g[i].x, x[j].y, acci[i][j]);
          acci[i][j] = fmaf(g[i].y, x[j].x, acci[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) Xn[(ty + 16 * i) * kN + tx + 32 * j] = cf{accr[i][j], acci[i][j]};
    __syncthreads();
    unsigned tmask = 0;                                    // fused: transposed rows' blocks
    if (dir == 0 && fused)
      for (int col = 0; col < 2; ++col)
        if ((active & (1u << col)) && ys[col] < L) tmask |= 1u << col;
    if (active) emit(Xn, k, active, tmask);
    if (dir == 0) {
      for (int col = 0; col < 2; ++col) {
        if (!(active & (1u << col))) continue;
        const int y = ys[col];
        if (y < L && !fused) {
          // rows (k, a) towards the column's start slice m = y: eta_{m,b} |G_{k,m}[a][b]|^2
          const float* em = eta + y * kW;
          float* dst = wt + (uint64_t)k * kW * K + (uint64_t)y * kW;
          for (int i = tid; i < kW * kW; i += kThreads) {
            const int a = i / kW, b = i % kW;               // b consecutive: coalesced rows
            dst[(uint64_t)a * K + b] = wsq(em[b], Xn[a * kN + col * kW + b]);
          }
        } else if (y == L + 1) {
          // lead-R weights of the rows of slice k from (G Phi_R)_k: eight threads per row
          const int a = tid >> 3, q = tid & 7;
          float part = 0.f;
#pragma unroll 4
          for (int nu = q * 8; nu < q * 8 + 8; ++nu) {
            const cf v = Xn[a * kN + col * kW + nu];
            part += (float)gam[d.lead_off + nu] * (v.x * v.x + v.y * v.y);
          }
          part += __shfl_xor_sync(0xffffffffu, part, 1);
          part += __shfl_xor_sync(0xffffffffu, part, 2);
          part += __shfl_xor_sync(0xffffffffu, part, 4);
          if (q == 0) {
            if (fused) l1[(uint64_t)(k * kW + a) * (L + 2) + L + 1] = part;
            else wt[(uint64_t)(k * kW + a) * K + n + 1] = part;
          }
        }
      }
    }
    cf* tmp = Xc;
    Xc = Xn;
    Xn = tmp;
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(err, ERR_NONFINITE);
}

// ---- 16 < W <= 32: the same recursion with the pair's 2W columns side by side --------------
// One CTA of 128 threads per job (four CTAs fit an SM): X_k [W][2W] = (-t g_k) [W][W] X_{k+1}
// in shared memory, thread (ty, tx) = (t / 16, t mod 16) owning the outputs a = ty + 8 i,
// b' = tx + 16 j.  g_{k-1} (or g_{k+1}) comes into registers while step k multiplies, so the
// step's only wait on global memory is hidden behind its products.
constexpr int kNThreads = 128;
constexpr int kNMax = 32;
constexpr size_t kNSmem = sizeof(cf) * (kNMax * kNMax + 2 * kNMax * 2 * kNMax) +
                          sizeof(float) * 2 * kNMax * (kNMax + 1);

template <int W>
__device__ __forceinline__ void chain_cta_narrow_body(const TaskDesc& d, const TcJob& job,
                                                      const float* __restrict__ eta32,
                                                      const float* __restrict__ phi32,
                                                      const double* __restrict__ gam,
                                                      const cf* __restrict__ gL,
                                                      const cf* __restrict__ gR,
                                                      const cf* __restrict__ start,
                                                      float* __restrict__ weights,
                                                      unsigned char* smem) {
  constexpr int N = 2 * W;                    // the pair's columns
  constexpr int RI = (W + 7) / 8;             // output rows a = ty + 8 i
  constexpr int CJ = (N + 15) / 16;           // output columns b' = tx + 16 j
  constexpr int WP = W + 1;                   // padded row of the weight staging
  constexpr int kPre = (W * W + kNThreads - 1) / kNThreads;
  cf* Gs = reinterpret_cast<cf*>(smem);                    // [a][c] (-t g_k); Phi at the edges
  cf* Xa = Gs + kNMax * kNMax;                             // [c][b'] ping
  cf* Xb = Xa + 2 * kNMax * kNMax;                         // [c][b'] pong
  float* Wt = reinterpret_cast<float*>(Xb + 2 * kNMax * kNMax);   // [b'][a] weights staging

  const int tid = threadIdx.x;
  const int L = d.L, n = d.n, K = d.K;
  const int dir = job.dir;
  auto m0_of = [&](int yy) { return yy < L ? yy : (yy == L ? 0 : L - 1); };
  const int ys[2] = {job.y0, job.y1};
  const float mt = (float)(-d.t);
  const float* eta = eta32 + d.onsite_off / 2;
  const cf* gsrc = (dir == 0 ? gL : gR) + d.g_off;
  float* wt = weights + d.wt_off;
  auto row_of = [&](int y, int b) -> uint64_t {
    return y < L ? (uint64_t)y * W + b : (uint64_t)n + (uint64_t)(y - L) * W + b;
  };
  auto load_start = [&](cf* X, int col) {
    const cf* st = start + d.start_off + (uint64_t)ys[col] * W * W;
    for (int i = tid; i < W * W; i += kNThreads) {
      const int c = i / W, b = i - c * W;
      X[c * N + col * W + b] = st[i];
    }
  };
  auto emit = [&](const cf* X, int k, unsigned mask) {
    for (int i = tid; i < N * W; i += kNThreads) {
      const int a = i / N, r = i - a * N;                  // r consecutive across threads
      const cf v = X[a * N + r];
      Wt[r * WP + a] = eta[k * W + a] * (v.x * v.x + v.y * v.y);
    }
    __syncthreads();
    for (int i = tid; i < N * W; i += kNThreads) {
      const int r = i / W, a = i - r * W;                  // a consecutive: coalesced rows
      const int col = r / W;
      if (mask & (1u << col))
        wt[row_of(ys[col], r - col * W) * K + (uint64_t)k * W + a] = Wt[r * WP + a];
    }
    if (k == 0 || k == L - 1) {
      // lead weights sum_nu Gamma_nu |(Phi^T X)_nu b'|^2: Phi (FP32) staged in Gs, free outside
      // the product; two threads per column, each half of the modes
      float* phis = reinterpret_cast<float*>(Gs);
      float* gams = phis + W * W;
      __syncthreads();
      for (int i = tid; i < W * W; i += kNThreads) phis[i] = phi32[d.phi_off + i];
      for (int i = tid; i < W; i += kNThreads) gams[i] = (float)gam[d.lead_off + i];
      __syncthreads();
      const int r = tid % 64, h = tid / 64;
      if (r < N) {
        float part = 0.f;
        for (int nu = h * (W / 2); nu < (h ? W : W / 2); ++nu) {
          float zr = 0.f, zi = 0.f;
#pragma unroll 8
          for (int a = 0; a < W; ++a) {
            const float p = phis[a * W + nu];
            const cf v = X[a * N + r];
            zr += p * v.x;
            zi += p * v.y;
          }
          part += gams[nu] * (zr * zr + zi * zi);
        }
        Wt[r * WP + h] = part;                             // staging is free again
      }
      __syncthreads();
      if (h == 0 && r < N) {
        const int col = r / W;
        if (mask & (1u << col)) {
          const float lw = Wt[r * WP] + Wt[r * WP + 1];
          const uint64_t base = row_of(ys[col], r - col * W) * K + n;
          if (k == 0) wt[base] = lw;
          if (k == L - 1) wt[base + 1] = lw;
        }
      }
    }
    __syncthreads();
  };

  unsigned have = 0;
  for (int col = 0; col < 2; ++col)
    if (ys[col] >= 0) have |= 1u << col;
  if (dir == 0) {
    for (int col = 0; col < 2; ++col) {
      if (!(have & (1u << col))) continue;
      load_start(Xa, col);
      __syncthreads();
      emit(Xa, m0_of(ys[col]), 1u << col);
    }
  }
  const int m0a = m0_of(job.y0), m0b = job.y1 >= 0 ? m0_of(job.y1) : m0a;
  const int k_first = dir == 0 ? max(m0a, m0b) - 1 : min(m0a, m0b) + 1;
  const int k_end = dir == 0 ? -1 : L;
  const int kstep = dir == 0 ? -1 : 1;
  cf gp[kPre];
  auto fetch = [&](int k) {
    const cf* gk = gsrc + (uint64_t)k * W * W;
#pragma unroll
    for (int r = 0; r < kPre; ++r) {
      const int i = tid + kNThreads * r;
      if (i < W * W) gp[r] = gk[i];
    }
  };
  if (k_first != k_end) fetch(k_first);
  cf* Xc = Xa;
  cf* Xn = Xb;
  const int ty = tid / 16, tx = tid % 16;
  for (int k = k_first; k != k_end; k += kstep) {
    unsigned active = 0;
    for (int col = 0; col < 2; ++col) {
      if (!(have & (1u << col))) continue;
      const int m0 = m0_of(ys[col]);
      if (dir == 0 ? k < m0 : k > m0) active |= 1u << col;
      if (dir == 0 ? k == m0 - 1 : k == m0 + 1) load_start(Xc, col);
    }
#pragma unroll
    for (int r = 0; r < kPre; ++r) {
      const int i = tid + kNThreads * r;
      if (i < W * W) Gs[i] = cf{mt * gp[r].x, mt * gp[r].y};
    }
    __syncthreads();
    if (k + kstep != k_end) fetch(k + kstep);
    float accr[RI][CJ], acci[RI][CJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) accr[i][j] = acci[i][j] = 0.f;
    // rows a >= W and columns b' >= N read in-bounds shared memory (a < 32, c N + b' < 64 W)
    // and are never stored
#pragma unroll 4
    for (int c = 0; c < W; ++c) {
      cf g[RI], x[CJ];
#pragma unroll
      for (int i = 0; i < RI; ++i) g[i] = Gs[(ty + 8 * i) * W + c];
#pragma unroll
      for (int j = 0; j < CJ; ++j) x[j] = Xc[c * N + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          accr[i][j] = fmaf(g[i].x, x[j].x, accr[i][j]);
          accr[i][j] = fmaf(-g[i].y, x[j].y, accr[i][j]);
          acci[i][j] = fmaf(g[i].x, x[j].y, acci[i][j]);
          acci[i][j] = fmaf(g[i].y, x[j].x, acci[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        const int a = ty + 8 * i, b = tx + 16 * j;
        if ((RI * 8 == W || a < W) && (CJ * 16 == N || b < N))
          Xn[a * N + b] = cf{accr[i][j], acci[i][j]};
      }
    __syncthreads();
    if (active) emit(Xn, k, active);
    cf* tmp = Xc;
    Xc = Xn;
    Xn = tmp;
  }
}

__global__ void __launch_bounds__(kNThreads, 4) chain_cta_narrow_kernel(
    const TaskDesc* __restrict__ tasks, const TcJob* __restrict__ jobs,
    const float* __restrict__ eta32, const float* __restrict__ phi32,
    const double* __restrict__ gam, const cf* __restrict__ gL, const cf* __restrict__ gR,
    const cf* __restrict__ start, float* __restrict__ weights) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TcJob job = jobs[blockIdx.x];
  const TaskDesc d = tasks[job.task];
#define NEGF_CN_CASE(w)                                                                       \
  case w:                                                                                     \
    chain_cta_narrow_body<w>(d, job, eta32, phi32, gam, gL, gR, start, weights, smem);        \
    break;
  switch (d.W) {
    NEGF_CN_CASE(17) NEGF_CN_CASE(18) NEGF_CN_CASE(19) NEGF_CN_CASE(20)
    NEGF_CN_CASE(21) NEGF_CN_CASE(22) NEGF_CN_CASE(23) NEGF_CN_CASE(24)
    NEGF_CN_CASE(25) NEGF_CN_CASE(26) NEGF_CN_CASE(27) NEGF_CN_CASE(28)
    NEGF_CN_CASE(29) NEGF_CN_CASE(30) NEGF_CN_CASE(31) NEGF_CN_CASE(32)
    default: break;
  }
#undef NEGF_CN_CASE
}

}  // namespace

cudaError_t launch_chain_cta(const TaskDesc* d_tasks, const TcJob* d_jobs, uint32_t n_wide,
                             uint32_t n_narrow, const float* d_eta32, const float* d_phi32,
                             const double* d_gam, const void* d_gL, const void* d_gR,
                             const void* d_start, void* d_weights, uint64_t* d_tab,
                             int32_t* d_err, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (n_wide) {
    e = cudaFuncSetAttribute(chain_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmem);
    if (e != cudaSuccess) return e;
    chain_cta_kernel<<<n_wide, kThreads, kSmem, s>>>(
        d_tasks, d_jobs, d_eta32, d_phi32, d_gam, static_cast<const cf*>(d_gL),
        static_cast<const cf*>(d_gR), static_cast<const cf*>(d_start),
        static_cast<float*>(d_weights), d_tab, d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (n_narrow) {
    e = cudaFuncSetAttribute(chain_cta_narrow_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNSmem);
    if (e != cudaSuccess) return e;
    chain_cta_narrow_kernel<<<n_narrow, kNThreads, kNSmem, s>>>(
        d_tasks, d_jobs + n_wide, d_eta32, d_phi32, d_gam, static_cast<const cf*>(d_gL),
        static_cast<const cf*>(d_gR), static_cast<const cf*>(d_start),
        static_cast<float*>(d_weights));
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace negf
