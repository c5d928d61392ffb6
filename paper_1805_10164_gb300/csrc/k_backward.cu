// Gradient of the Monte Carlo transmission w.r.t. onsite energies and dephasing.
//
// The paper does not differentiate its estimator.  Per task the walk estimates
// T = c_p P(q|p) with c_p = sum_m u_m (Eq. elast_lin_xpq, Eq. lead_out_probability), and a walk
// is a path m -> a_1 -> ... -> lead drawn with probability (u_m / c_p) prod P_ab, P_ab = w_ab /
// rowsum_a.  The score-function identity d E[1_q] = E[(1_q - b) d log p(path)] (any constant b;
// b = P_hat makes the injection term's c_p part vanish) gives, from the score tallies
// C^r_ab = number of a -> b transitions on walks absorbed at r,
//   s_ab = (C^q_ab - P_hat (C^L_ab + C^R_ab)) / N,     s_m likewise for the injection modes,
//   dT  = sum_m (P_hat + c_p s_m / u_m) du_m + c_p sum_ab (s_ab / w_ab - S_a / rowsum_a) dw_ab,
// S_a = sum_b s_ab.  The weights depend on G = (E - H - Sigma)^{-1}; with Gbar the Wirtinger
// seed of every G element (dT = 2 Re sum Gbar_ij dG_ij) and dG = G e_k e_k^T G for V_k,
// dG = -(i/2) G e_k e_k^T G for eta_k:
//   dT/dV_k = 2 Re (G Gbar G)_kk,   dT/deta_k = Im (G Gbar G)_kk + (explicit gamma_k terms).
// Kernels: seeds (one warp per table row), Gbar assembly (site, lead, injection and mode
// terms in separate passes so no two threads add to one element), Y = Gbar G (tiled complex
// GEMM), the diagonal of G Y, and the per-wire sums weighted by w_E (f_p - f_q).
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

template <typename C> struct RealOf;
template <> struct RealOf<cd> { using T = double; };
template <> struct RealOf<cf> { using T = float; };
__device__ __forceinline__ cd conjc(cd a) { return cd{a.x, -a.y}; }
__device__ __forceinline__ cf conjc(cf a) { return cf{a.x, -a.y}; }

// ---- seeds: wbar_ab = c_p (s_ab / w_ab - S_a / rowsum_a) for every row; one warp per row.
// Injection-mode seeds ubar_m = P_hat + c_p s_m / u_m (rows = rows + 2 jobs per task: the last
// two are the mode rows).  The seeds are formed in FP64 and stored as Wo (FP64, or FP32 for the
// block-column adjoint of FP32 tables, which forms its products in FP32).
template <typename R, typename Wo>
__global__ void seeds_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs,
                             const R* __restrict__ weights, const double* __restrict__ rowsum,
                             const double* __restrict__ mode_w, const double* __restrict__ cvals,
                             const unsigned long long* __restrict__ counts,
                             const unsigned long long* __restrict__ score, uint64_t stride,
                             const unsigned long long* __restrict__ mode_score,
                             uint32_t mode_stride, int p, Wo* __restrict__ wbar,
                             double* __restrict__ ubar) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t job = blockIdx.x * (blockDim.x >> 5) + warp;
  if (job >= n_jobs) return;
  int lo = 0, hi = n_tasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].row_base <= job) lo = mid; else hi = mid - 1;
  }
  const int task = lo;
  const TaskDesc& d = tasks[task];
  const int q = 1 - p;
  const unsigned long long* tc = counts + (size_t)task * NEGF_TALLY_FIELDS;
  const double N = (double)tc[0];
  const double Ph = N > 0.0 ? (double)tc[1 + q] / N : 0.0;
  const double c = cvals[2 * task + p];
  const int row = (int)(job - d.row_base);
  if (row < d.rows) {
    const int K = d.K;
    const uint64_t off = d.wt_off + (uint64_t)row * K;
    const unsigned long long* C0 = score + off;
    const unsigned long long* C1 = score + stride + off;
    // The FP64 pipe of this GPU is narrow: 1/N and S/rowsum once per row; S from the row's
    // integer count sums (exact): with s_ab = (Cq - Ph (C0 + C1)) / N,
    // S = (sum Cq - Ph (sum C0 + sum C1)) / N
    const double invN = N > 0.0 ? 1.0 / N : 0.0;
    unsigned long long sq = 0, s01 = 0;
    for (int b = lane; b < K; b += 32) {
      const unsigned long long c0 = C0[b], c1 = C1[b];
      sq += q == 0 ? c0 : c1;
      s01 += c0 + c1;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
      s01 += __shfl_xor_sync(0xffffffffu, s01, o);
    }
    const double S = ((double)sq - Ph * (double)s01) * invN;
    const double rs = rowsum[d.row_base + row];
    const double Srs = rs > 0.0 ? S / rs : 0.0;
    // wbar = c (s / w - S / rs) = (c / N) (Cq - Ph (C0 + C1)) / w - c S / rs
    const double cN = c * invN, cS = c * Srs;
    for (int b = lane; b < K; b += 32) {
      const unsigned long long c0 = C0[b], c1 = C1[b];
      const double D = fma(-Ph, (double)(c0 + c1), (double)(q == 0 ? c0 : c1));
      double v = 0.0;
      if (sizeof(R) == 4) {
        // FP32 weight w: 1/w from the FP32 reciprocal and one Newton step in FP64
        // (r <- r + r (1 - w r): relative error ~2^-46, far below the FP32 table bar); weights
        // whose reciprocal leaves the normal FP32 range are divided in FP64
        const float wf = (float)weights[off + b];
        if (wf > 0.f) {
          const double wv = (double)wf;
          if (wf >= 0x1p-125f && wf <= 0x1p125f) {
            double r = (double)__frcp_rn(wf);
            r = fma(r, fma(-wv, r, 1.0), r);
            v = D * r;
          } else {
            v = D / wv;
          }
        }
      } else {
        const double wv = (double)weights[off + b];
        if (wv > 0.0) v = D / wv;
      }
      wbar[off + b] = (Wo)fma(cN, v, -cS);
    }
  } else if (row == d.rows) {
    // injection modes of the start lead p (W up to 64: two per lane)
    for (int m = lane; m < d.W; m += 32) {
      const uint32_t mo = d.mode_off + p * d.W + m;
      const double u = mode_w[mo];
      const double C0 = (double)mode_score[mo], C1 = (double)mode_score[mode_stride + mo];
      const double Cq = q == 0 ? C0 : C1;
      const double s = N > 0.0 ? (Cq - Ph * (C0 + C1)) / N : 0.0;
      ubar[d.mode_off + p * d.W + m] = Ph + (u > 0.0 ? c * s / u : 0.0);
    }
  }
}

// ---- Gbar assembly for one task (dense n x n, row-major, element (i, j)).
// Pass A: site rows a, site columns b: Gbar[b][a] = wbar_ab gamma_b conj(G[b][a]).
template <typename C>
__global__ void gbar_sites_kernel(TaskDesc d, const C* __restrict__ G,
                                  const double* __restrict__ wbar, const double* __restrict__ eta,
                                  C* __restrict__ Gbar) {
  using R = typename RealOf<C>::T;
  const int n = d.n, K = d.K;
  const uint64_t total = (uint64_t)n * n;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / n), a = (int)(idx % n);      // element (b, a)
    const R s = (R)(wbar[d.wt_off + (uint64_t)a * K + b] * eta[b]);
    const C g = conjc(G[idx]);
    Gbar[idx] = C{s * g.x, s * g.y};
  }
}

// Pass B: lead columns of the site rows: for row a and lead r, y_nu = sum_x phi_nu(x)
// G[(r,x)][a]; Gbar[(r,x)][a] += wbar_{a,n+r} sum_nu Gamma_nu phi_nu(x) conj(y_nu).
// A CTA takes 256 / W sites a: thread (a, q) first forms y_q of its site (shared memory), then
// the Gbar element of x = q, so that y is formed once per site rather than once per (a, x).
// The two leads are done one after the other (L = 1 puts both on slice 0, so they must not
// run concurrently).
template <typename C>
__global__ void __launch_bounds__(256) gbar_leads_kernel(TaskDesc d, const C* __restrict__ G,
                                                         const double* __restrict__ wbar,
                                                         const double* __restrict__ phi,
                                                         const double* __restrict__ gam,
                                                         C* __restrict__ Gbar, int r) {
  using R = typename RealOf<C>::T;
  __shared__ double sy[256][2];
  const int n = d.n, W = d.W, K = d.K;
  const int k0 = (r == 0 ? 0 : d.L - 1) * W;
  const int per = 256 / W;                       // sites per CTA (W <= 64)
  const int t = threadIdx.x, al = t / W, q = t - al * W;
  const int a = blockIdx.x * per + al;
  const bool live = al < per && a < n;
  const double wb = live ? wbar[d.wt_off + (uint64_t)a * K + n + r] : 0.0;
  if (wb != 0.0) {
    double yx = 0.0, yy = 0.0;
    for (int xx = 0; xx < W; ++xx) {
      const C g = G[(uint64_t)(k0 + xx) * n + a];
      yx += phi[xx * W + q] * (double)g.x;
      yy += phi[xx * W + q] * (double)g.y;
    }
    sy[t][0] = yx;
    sy[t][1] = yy;
  }
  __syncthreads();
  if (wb != 0.0) {
    double tx = 0.0, ty = 0.0;
    for (int nu = 0; nu < W; ++nu) {
      const double f = gam[nu] * phi[q * W + nu];
      tx += f * sy[al * W + nu][0];
      ty -= f * sy[al * W + nu][1];                  // conj(y)
    }
    C* o = Gbar + (uint64_t)(k0 + q) * n + a;
    o->x += (R)(wb * tx);
    o->y += (R)(wb * ty);
  }
}

// Pass C: injection rows (p, m): psi = G Phi_p[:, m] (gphi), psibar_b = wbar gamma_b conj(psi_b)
// for sites, plus the lead-column terms on the boundary slices; then
// Gbar[b][(p,y)] += sum_m psibar^(m)_b phi_m(y).  One thread per (b, y).
// The lead-column term of injection row m at site x of the boundary slice sr (lead r) is
// wbar_{(p,m),n+r} Tl[r][m][x], with z_nu = sum_x' phi_nu(x') psi_(sr,x') and
// Tl[r][m][x] = sum_nu Gamma_nu phi_nu(x) conj(z_nu): it depends on neither the column y nor
// the other sites, so gbar_inj_lead_kernel forms it once (one CTA per (r, m), z in shared
// memory) before the per-element pass.  Tl: [nr][W][W] in the precision of G (nr = 1 when
// L = 1: both leads then sit on slice 0 and share it).
template <typename C>
__global__ void gbar_inj_lead_kernel(TaskDesc d, const C* __restrict__ gphi,
                                     const double* __restrict__ phi,
                                     const double* __restrict__ gam, int p, C* __restrict__ Tl) {
  __shared__ double sz[2 * 64];
  const int W = d.W, L = d.L;
  const int r = blockIdx.x / W, m = blockIdx.x % W;
  const int sr = r == 0 ? 0 : L - 1;
  for (int nu = threadIdx.x; nu < W; nu += blockDim.x) {
    double zx = 0.0, zy = 0.0;
    for (int xx = 0; xx < W; ++xx) {
      const C g = gphi[(uint64_t)(sr * W + xx) * 2 * W + p * W + m];
      zx += phi[xx * W + nu] * (double)g.x;
      zy += phi[xx * W + nu] * (double)g.y;
    }
    sz[2 * nu] = zx;
    sz[2 * nu + 1] = zy;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    double tx = 0.0, ty = 0.0;
    for (int nu = 0; nu < W; ++nu) {
      const double f = gam[nu] * phi[x * W + nu];
      tx += f * sz[2 * nu];
      ty -= f * sz[2 * nu + 1];
    }
    using R = typename RealOf<C>::T;
    Tl[((uint64_t)r * W + m) * W + x] = C{(R)tx, (R)ty};
  }
}

template <typename C>
__global__ void gbar_inj_kernel(TaskDesc d, const C* __restrict__ gphi,
                                const double* __restrict__ wbar, const double* __restrict__ eta,
                                const double* __restrict__ phi, const C* __restrict__ Tl, int p,
                                C* __restrict__ Gbar) {
  using R = typename RealOf<C>::T;
  const int n = d.n, W = d.W, K = d.K, L = d.L;
  const int total = n * W;
  const int kp = (p == 0 ? 0 : L - 1) * W;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int b = idx / W, y = idx % W;
    const int sb = b / W, xb = b % W;                         // slice and row of site b
    double ax = 0.0, ay = 0.0;
    for (int m = 0; m < W; ++m) {
      const uint64_t roff = d.wt_off + (uint64_t)(n + p * W + m) * K;
      const C ps = gphi[(uint64_t)b * 2 * W + p * W + m];
      double bx = wbar[roff + b] * eta[b] * (double)ps.x;     // psibar_b = wbar gamma conj(psi)
      double by = -wbar[roff + b] * eta[b] * (double)ps.y;
      for (int r = 0; r < 2; ++r) {
        const int sr = r == 0 ? 0 : L - 1;
        if (sb != sr) continue;
        const double wl = wbar[roff + n + r];
        if (wl == 0.0) continue;
        const C t = Tl[((uint64_t)(L == 1 ? 0 : r) * W + m) * W + xb];
        bx += wl * (double)t.x;
        by += wl * (double)t.y;
      }
      ax += bx * phi[y * W + m];
      ay += by * phi[y * W + m];
    }
    C* o = Gbar + (uint64_t)b * n + kp + y;
    o->x += (R)ax;
    o->y += (R)ay;
  }
}

// Pass D: mode weights u_m = lambda_m <phi_m|A|phi_m> = -2 lambda_m Im(phi_m^T G phi_m):
// Gbar[(p,x)][(p,y)] += i ubar_m lambda_m phi_m(x) phi_m(y).
template <typename C>
__global__ void gbar_modes_kernel(TaskDesc d, const double* __restrict__ ubar,
                                  const double* __restrict__ phi, const double* __restrict__ gam,
                                  int p, C* __restrict__ Gbar) {
  using R = typename RealOf<C>::T;
  const int n = d.n, W = d.W;
  const int kp = (p == 0 ? 0 : d.L - 1) * W;
  for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
    const int x = idx / W, y = idx % W;
    double v = 0.0;
    for (int m = 0; m < W; ++m)
      v += ubar[d.mode_off + p * W + m] * gam[m] * phi[x * W + m] * phi[y * W + m];
    C* o = Gbar + (uint64_t)(kp + x) * n + kp + y;
    o->y += (R)v;
  }
}

// ---- Y = A B for dense complex n x n (row-major), tiled in shared memory: a 64 x 64 block of
// Y per CTA, k in steps of 16; thread (ty, tx) of 16 x 16 owns rows ty + 16 i and columns
// tx + 16 j (i, j < 4), so that each k costs 8 shared loads for 16 complex multiply-adds.  The
// A tile is kept transposed ([k][row]) so that a warp's row loads are broadcasts.
constexpr int kGemmM = 64, kGemmK = 16;

template <typename C>
__global__ void __launch_bounds__(256) cgemm_kernel(const C* __restrict__ A,
                                                    const C* __restrict__ B, C* __restrict__ Y,
                                                    int n) {
  using R = typename RealOf<C>::T;
  __shared__ C sA[kGemmK][kGemmM + 1];
  __shared__ C sB[kGemmK][kGemmM];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.y * kGemmM, col0 = blockIdx.x * kGemmM;
  R accr[4][4], acci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = (R)0;
  for (int k0 = 0; k0 < n; k0 += kGemmK) {
    // A tile: 64 rows x 16 k (row r = e / 16, k = e % 16: 16 consecutive k of a row per
    // half-warp); B tile: 16 k x 64 columns (consecutive columns per warp)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int ar = e >> 4, ak = e & 15;
      const int gr = row0 + ar, gk = k0 + ak;
      sA[ak][ar] = (gr < n && gk < n) ? A[(uint64_t)gr * n + gk] : C{0, 0};
      const int bk = e >> 6, bc = e & 63;
      const int hk = k0 + bk, hc = col0 + bc;
      sB[bk][bc] = (hk < n && hc < n) ? B[(uint64_t)hk * n + hc] : C{0, 0};
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGemmK; ++k) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] += a[i].x * b[j].x - a[i].y * b[j].y;
          acci[i][j] += a[i].x * b[j].y + a[i].y * b[j].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < n && c < n) Y[(uint64_t)r * n + c] = C{accr[i][j], acci[i][j]};
    }
}

// ---- dT/dV_k = 2 Re (G Y)_kk, dT/deta_k = Im (G Y)_kk + explicit gamma_k terms:
// sum over rows of wbar_{row,k} |.|^2 where |.|^2 = |G[k][a]|^2 (site rows a) or |psi_m,k|^2.
// One warp per k.
template <typename C>
__global__ void grad_diag_kernel(TaskDesc d, const C* __restrict__ G, const C* __restrict__ Y,
                                 const C* __restrict__ gphi, const double* __restrict__ wbar,
                                 double* __restrict__ dV, double* __restrict__ dEta) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + warp;
  const int n = d.n, K = d.K, W = d.W;
  if (k >= n) return;
  double zx = 0.0, zy = 0.0, ex = 0.0;
  for (int i = lane; i < n; i += 32) {
    const C g = G[(uint64_t)k * n + i];
    const C y = Y[(uint64_t)i * n + k];
    zx += (double)g.x * y.x - (double)g.y * y.y;
    zy += (double)g.x * y.y + (double)g.y * y.x;
    ex += wbar[d.wt_off + (uint64_t)i * K + k] * ((double)g.x * g.x + (double)g.y * g.y);
  }
  for (int j = lane; j < 2 * W; j += 32) {
    const C ps = gphi[(uint64_t)k * 2 * W + j];
    ex += wbar[d.wt_off + (uint64_t)(n + j) * K + k] * ((double)ps.x * ps.x + (double)ps.y * ps.y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    zx += __shfl_down_sync(0xffffffffu, zx, o);
    zy += __shfl_down_sync(0xffffffffu, zy, o);
    ex += __shfl_down_sync(0xffffffffu, ex, o);
  }
  if (lane == 0) {
    dV[k] = 2.0 * zx;
    dEta[k] = zy + ex;
  }
}

// ---- dI/dtheta per wire: sum over the wire's tasks (fixed order) of
// seed_w * w_E (f_p - f_q) dT/dtheta.  One thread per (wire, site).
__device__ __forceinline__ double fermi_b(double E, double mu, double kT) {
  return 0.5 * (1.0 - tanh(0.5 * (E - mu) / kT));
}

__global__ void grad_sum_kernel(const TaskDesc* __restrict__ tasks, int n_wires,
                                const int32_t* __restrict__ wire_task0,
                                const uint64_t* __restrict__ task_site_off,
                                const uint64_t* __restrict__ wire_site_off,
                                const double* __restrict__ dT_V, const double* __restrict__ dT_E,
                                const double* __restrict__ seed, double mu_p, double mu_q,
                                double kT, double* __restrict__ out_V, double* __restrict__ out_E) {
  const int w = blockIdx.x;
  if (w >= n_wires) return;
  const int t0 = wire_task0[w], t1 = wire_task0[w + 1];
  if (t0 == t1) return;
  const int n = tasks[t0].n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double aV = 0.0, aE = 0.0;
    for (int t = t0; t < t1; ++t) {
      const TaskDesc& d = tasks[t];
      const double wd = seed[w] * d.w_E * (fermi_b(d.E, mu_p, kT) - fermi_b(d.E, mu_q, kT));
      aV += wd * dT_V[task_site_off[t] + k];
      aE += wd * dT_E[task_site_off[t] + k];
    }
    out_V[wire_site_off[w] + k] = aV;
    out_E[wire_site_off[w] + k] = aE;
  }
}

template <typename C>
cudaError_t backward_task(const TaskDesc& d, const C* G, const C* gphi, const double* wbar,
                          const double* ubar, const double* eta, const double* phi,
                          const double* gam, int p, C* Gbar, C* Y, double* dV, double* dE,
                          int sm_count, int32_t* err, cudaStream_t s) {
  const int n = d.n, W = d.W;
  const uint64_t nn = (uint64_t)n * n;
  unsigned blocks = (unsigned)((nn + 255) / 256);
  if (blocks > (unsigned)sm_count * 32) blocks = (unsigned)sm_count * 32;
  gbar_sites_kernel<C><<<blocks, 256, 0, s>>>(d, G, wbar, eta, Gbar);
  const unsigned bl = (unsigned)((n * W + 255) / 256);
  const unsigned bll = (unsigned)((n + 256 / W - 1) / (256 / W));
  gbar_leads_kernel<C><<<bll, 256, 0, s>>>(d, G, wbar, phi, gam, Gbar, 0);
  gbar_leads_kernel<C><<<bll, 256, 0, s>>>(d, G, wbar, phi, gam, Gbar, 1);
  // the lead terms of the injection rows go through Y, which the product below overwrites
  gbar_inj_lead_kernel<C><<<(d.L == 1 ? 1 : 2) * W, 64, 0, s>>>(d, gphi, phi, gam, p, Y);
  gbar_inj_kernel<C><<<bl, 256, 0, s>>>(d, gphi, wbar, eta, phi, Y, p, Gbar);
  gbar_modes_kernel<C><<<1, 256, 0, s>>>(d, ubar, phi, gam, p, Gbar);
  if constexpr (sizeof(C) == sizeof(cf)) {
    // complex64: the product on the tensor cores (3xTF32, FP32 accumulation)
    const cudaError_t e = launch_cgemm_tc(reinterpret_cast<const cf*>(Gbar),
                                          reinterpret_cast<const cf*>(G),
                                          reinterpret_cast<cf*>(Y), n, err, s);
    if (e != cudaSuccess) return e;
  } else {
    dim3 grid((n + kGemmM - 1) / kGemmM, (n + kGemmM - 1) / kGemmM);
    cgemm_kernel<C><<<grid, 256, 0, s>>>(Gbar, G, Y, n);
  }
  grad_diag_kernel<C><<<(n + 7) / 8, 256, 0, s>>>(d, G, Y, gphi, wbar, dV, dE);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward_seeds(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs,
                                  int precision, const void* d_weights, const double* d_rowsum,
                                  const double* d_mode_w, const double* d_c,
                                  const uint64_t* d_counts, const uint64_t* d_score,
                                  uint64_t stride, const uint64_t* d_mode_score,
                                  uint32_t mode_stride, int start_lead, void* d_wbar,
                                  int wbar_fp32, double* d_ubar, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  const unsigned blocks = (n_jobs + 7) / 8;
  const auto* cnt = reinterpret_cast<const unsigned long long*>(d_counts);
  const auto* sc = reinterpret_cast<const unsigned long long*>(d_score);
  const auto* ms = reinterpret_cast<const unsigned long long*>(d_mode_score);
  if (precision == NEGF_FP64)
    seeds_kernel<double, double><<<blocks, 256, 0, s>>>(
        d_tasks, n_tasks, n_jobs, static_cast<const double*>(d_weights), d_rowsum, d_mode_w, d_c,
        cnt, sc, stride, ms, mode_stride, start_lead, static_cast<double*>(d_wbar), d_ubar);
  else if (wbar_fp32)
    seeds_kernel<float, float><<<blocks, 256, 0, s>>>(
        d_tasks, n_tasks, n_jobs, static_cast<const float*>(d_weights), d_rowsum, d_mode_w, d_c,
        cnt, sc, stride, ms, mode_stride, start_lead, static_cast<float*>(d_wbar), d_ubar);
  else
    seeds_kernel<float, double><<<blocks, 256, 0, s>>>(
        d_tasks, n_tasks, n_jobs, static_cast<const float*>(d_weights), d_rowsum, d_mode_w, d_c,
        cnt, sc, stride, ms, mode_stride, start_lead, static_cast<double*>(d_wbar), d_ubar);
  return cudaGetLastError();
}

cudaError_t launch_backward_task(const TaskDesc& d, int precision, const void* G,
                                 const void* gphi, const double* wbar, const double* ubar,
                                 const double* eta, const double* phi, const double* gam,
                                 int start_lead, void* Gbar, void* Y, double* dV, double* dE,
                                 int sm_count, int32_t* d_err, cudaStream_t s) {
  if (precision == NEGF_FP64)
    return backward_task<cd>(d, static_cast<const cd*>(G), static_cast<const cd*>(gphi), wbar,
                             ubar, eta, phi, gam, start_lead, static_cast<cd*>(Gbar),
                             static_cast<cd*>(Y), dV, dE, sm_count, d_err, s);
  return backward_task<cf>(d, static_cast<const cf*>(G), static_cast<const cf*>(gphi), wbar,
                           ubar, eta, phi, gam, start_lead, static_cast<cf*>(Gbar),
                           static_cast<cf*>(Y), dV, dE, sm_count, d_err, s);
}

cudaError_t launch_grad_sum(const TaskDesc* d_tasks, int n_wires, const int32_t* d_wire_task0,
                            const uint64_t* d_task_site_off, const uint64_t* d_wire_site_off,
                            const double* dT_V, const double* dT_E, const double* d_seed,
                            double mu_p, double mu_q, double kT, double* out_V, double* out_E,
                            cudaStream_t s) {
  if (n_wires == 0) return cudaSuccess;
  grad_sum_kernel<<<n_wires, 256, 0, s>>>(d_tasks, n_wires, d_wire_task0, d_task_site_off,
                                          d_wire_site_off, dT_V, dT_E, d_seed, mu_p, mu_q, kT,
                                          out_V, out_E);
  return cudaGetLastError();
}

}  // namespace negf
