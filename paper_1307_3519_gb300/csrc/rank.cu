// rank.cu -- per-trait average-rank transform (section "Input data": ranks per
// trait row; section "Handling tied data": average ranks for ties and the factor
// sum(t^3 - t); section "Handling missing values": NaN samples are left out).
//
// One warp per trait.  The row is staged in shared memory and each present
// sample k counts lo = #{j present: x_j < x_k} and eq = #{j present: x_j == x_k}
// (k itself included), so 2 * average rank = 2 lo + eq + 1, exactly.  The stored
// value is the centred integer a = 2 lo + eq - K = 2 rank - (K + 1), |a| <= K-1,
// which FP16 holds exactly for K <= 512 (integers up to 2048 are exact).  The
// run containing k has length eq, so sum_k (eq_k^2 - 1) = sum_runs (t^3 - t).
#include "common.cuh"

namespace krux {

namespace {
constexpr int kRankWarps = 8;

// Tie factor C = 1 - sum(t^3-t)/(K^3-K) and the trait constants of the scan:
// H = 3/(K(K+1)C) * sum_i D_i^2/N_i, so cfac = 3/(K(K+1)C) and the fast-test
// bound tau = K(K+1)C/3; degenerate traits (K < 2 or C = 0) get cfac 0, tau +inf.
__device__ __forceinline__ void trait_consts(int K, long long tie, float &tau, double &cfac) {
  const double Kd = (double)K;
  const double C = K >= 2 ? 1.0 - (double)tie / (Kd * Kd * Kd - Kd) : 0.0;
  if (K >= 2 && C > 0.0) {
    const double s = Kd * (Kd + 1.0) * C;
    cfac = 3.0 / s;
    tau = (float)(s / 3.0);
  } else {
    cfac = 0.0;
    tau = __int_as_float(0x7f800000);  // +inf: never a hit
  }
}

__global__ void __launch_bounds__(kRankWarps * 32)
rank_kernel(const float *__restrict__ expr, int T, int N, int64_t ld, int Np, RankDev r) {
  extern __shared__ float srow[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kRankWarps + warp;
  if (t >= T) return;  // whole warp leaves together; no block-level barrier follows
  float *x = srow + warp * N;
  const float *row = expr + (int64_t)t * ld;
  for (int k = lane; k < N; k += 32) x[k] = row[k];
  __syncwarp();

  // present count and the list of NaN samples, in sample order
  int K = 0, nan_seen = 0;
  for (int k0 = 0; k0 < N; k0 += 32) {
    const int k = k0 + lane;
    const bool isn = (k < N) && isnan(x[k]);
    const bool pres = (k < N) && !isn;
    const unsigned bn = __ballot_sync(0xffffffffu, isn);
    K += __popc(__ballot_sync(0xffffffffu, pres));
    if (isn) r.nan_idx[(int64_t)t * N + nan_seen + __popc(bn & ((1u << lane) - 1u))] = (uint16_t)k;
    nan_seen += __popc(bn);
  }

  long long tie = 0;
  for (int k = lane; k < Np; k += 32) {
    int a = 0;
    if (k < N) {
      const float xk = x[k];
      uint16_t lo16 = 0, eq16 = 0;
      if (!isnan(xk)) {
        int lo = 0, eq = 0;
        int j = 0;
        for (; j + 4 <= N; j += 4) {
          const float x0 = x[j], x1 = x[j + 1], x2 = x[j + 2], x3 = x[j + 3];
          lo += (x0 < xk) + (x1 < xk) + (x2 < xk) + (x3 < xk);
          eq += (x0 == xk) + (x1 == xk) + (x2 == xk) + (x3 == xk);
        }
        for (; j < N; ++j) {
          lo += (x[j] < xk);
          eq += (x[j] == xk);
        }
        lo16 = (uint16_t)lo;
        eq16 = (uint16_t)eq;
        tie += (long long)eq * eq - 1;
        a = 2 * lo + eq - K;
      }
      r.lo[(int64_t)t * N + k] = lo16;
      r.eq[(int64_t)t * N + k] = eq16;
    }
    r.A[(int64_t)t * Np + k] = __int2half_rn(a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tie += __shfl_xor_sync(0xffffffffu, tie, o);

  if (lane == 0) {
    r.tie[t] = tie;
    r.K[t] = K;
    r.nan_cnt[t] = (uint16_t)(N - K);
    if (N - K > 0) atomicMax(&r.tile_nan[t / kTileM], (uint32_t)(N - K));
  }
}

// out[p][row][k] = A[row][perm_p[k]] for k < N (padding columns stay 0): the
// rank matrix of the expression with its sample columns permuted (ranks, tie
// sums and K are invariant under a column permutation).
__global__ void permute_rows_kernel(const __half *__restrict__ A, __half *__restrict__ out,
                                    int rows_pad, int Np, int N, const int32_t *__restrict__ perms,
                                    int P, unsigned int *status) {
  const int64_t total = (int64_t)P * rows_pad * Np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % Np);
    const int64_t pr = i / Np;
    const int row = (int)(pr % rows_pad);
    const int p = (int)(pr / rows_pad);
    __half v = __int2half_rn(0);
    if (k < N) {
      const int32_t src = perms[(int64_t)p * N + k];
      if (src >= 0 && src < N)
        v = A[(int64_t)row * Np + src];
      else if (status != nullptr)
        atomicOr(status, kDevBadPerm);
    }
    out[i] = v;
  }
}
// inv[q][perms[q][k]] = k (entries outside 0..N-1 are skipped; the row gather
// reports them).
__global__ void invert_perms_kernel(const int32_t *__restrict__ perms, int P, int N,
                                    int32_t *__restrict__ inv) {
  const int64_t total = (int64_t)P * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / N), k = (int)(i % N);
    const int32_t v = perms[i];
    if (v >= 0 && v < N) inv[(int64_t)q * N + v] = k;
  }
}

__global__ void permute_nan_idx_kernel(const uint16_t *__restrict__ nan_cnt,
                                       const uint16_t *__restrict__ nan_idx, int T, int N,
                                       const int32_t *__restrict__ inv, int P,
                                       uint16_t *__restrict__ out) {
  const int64_t total = (int64_t)P * T * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % N);
    const int64_t qt = i / N;
    const int t = (int)(qt % T);
    const int q = (int)(qt / T);
    if (j < nan_cnt[t]) out[i] = (uint16_t)inv[(int64_t)q * N + nan_idx[(int64_t)t * N + j]];
  }
}
}  // namespace

// Per-trait constants of the padding rows of the last 128-trait tile: never a hit.
__global__ void pad_traits_kernel(int T, int rows_pad, float *tau, double *cfac, uint16_t *nan_cnt) {
  const int t = T + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows_pad) return;
  tau[t] = __int_as_float(0x7f800000);
  cfac[t] = 0.0;
  nan_cnt[t] = 0;
}

// The FP64 trait constants of a rank set, one thread per row (FP64 issue is slow
// on this part; done by one lane per trait in rank_kernel they cost most of its
// time); padding rows get cfac 0, tau +inf and no NaN.
__global__ void __launch_bounds__(256) rank_consts_kernel(int T, int rows_pad, RankDev r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows_pad) return;
  if (t < T) {
    trait_consts(r.K[t], r.tie[t], r.tau[t], r.cfac[t]);
  } else {
    r.tau[t] = __int_as_float(0x7f800000);
    r.cfac[t] = 0.0;
    r.nan_cnt[t] = 0;
  }
}

cudaError_t launch_pad_traits(int T, int rows_pad, float *tau, double *cfac, uint16_t *nan_cnt,
                              cudaStream_t s) {
  if (rows_pad <= T) return cudaSuccess;
  pad_traits_kernel<<<1, 128, 0, s>>>(T, rows_pad, tau, cfac, nan_cnt);
  return cudaGetLastError();
}

cudaError_t launch_rank(const float *expr, int T, int N, int64_t ld, int Np, int rows_pad,
                        const RankDev &r, cudaStream_t s) {
  const int grid = (T + kRankWarps - 1) / kRankWarps;
  const size_t smem = (size_t)kRankWarps * N * sizeof(float);
  rank_kernel<<<grid, kRankWarps * 32, smem, s>>>(expr, T, N, ld, Np, r);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rank_consts_kernel<<<(rows_pad + 255) / 256, 256, 0, s>>>(T, rows_pad, r);
  return cudaGetLastError();
}

cudaError_t launch_invert_perms(const int32_t *perms, int P, int N, int32_t *inv, cudaStream_t s) {
  const int64_t total = (int64_t)P * N;
  if (total == 0) return cudaSuccess;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 4) grid = 152 * 4;
  invert_perms_kernel<<<grid, 256, 0, s>>>(perms, P, N, inv);
  return cudaGetLastError();
}

cudaError_t launch_permute_nan_idx(const uint16_t *nan_cnt, const uint16_t *nan_idx, int T, int N,
                                   const int32_t *inv, int P, uint16_t *out, cudaStream_t s) {
  const int64_t total = (int64_t)P * T * N;
  if (total == 0) return cudaSuccess;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  permute_nan_idx_kernel<<<grid, 256, 0, s>>>(nan_cnt, nan_idx, T, N, inv, P, out);
  return cudaGetLastError();
}

cudaError_t launch_permute_rows(const __half *A, __half *out, int rows_pad, int Np, int N,
                                const int32_t *perms, int P, unsigned int *status, cudaStream_t s) {
  const int64_t total = (int64_t)P * rows_pad * Np;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  permute_rows_kernel<<<grid, 256, 0, s>>>(A, out, rows_pad, Np, N, perms, P, status);
  return cudaGetLastError();
}

}  // namespace krux

// ---------------------------------------------------------------------------
// Ranks of every trait over the samples left after dropping a missing-genotype
// pattern (section "Handling missing values": a new expression matrix with the
// samples of the pattern removed, re-ranked).  No re-sort: for present samples,
// x_q < x_k exactly when lo_q < lo_k and x_q == x_k exactly when lo_q == lo_k,
// so lo' = lo - #{q dropped, present, lo_q < lo_k} and
// eq' = eq - #{q dropped, present, lo_q == lo_k}.  One launch re-ranks every
// bucket of a call (grid.y = bucket).
namespace krux {
namespace {
__global__ void __launch_bounds__(256)
rerank_kernel(const RerankJob *__restrict__ jobs, const int32_t *__restrict__ drops) {
  const RerankJob &J = jobs[blockIdx.y];
  const int N = J.N, Np = J.Np, T = J.T, n_drop = J.n_drop;
  __shared__ uint32_t dmask[kMaxN / 32];
  __shared__ int32_t dlist[kMaxN];
  for (int i = threadIdx.x; i < kMaxN / 32; i += blockDim.x) dmask[i] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < n_drop; i += blockDim.x) {
    const int q = drops[J.drop_off + i];
    dlist[i] = q;
    atomicOr(&dmask[q >> 5], 1u << (q & 31));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 8 + warp;
  if (t >= J.rows_pad) return;
  if (t >= T) {  // padding row (its constants come from rerank_consts_kernel)
    for (int k = lane; k < Np; k += 32) J.A[(int64_t)t * Np + k] = __int2half_rn(0);
    return;
  }
  const uint16_t *lo = J.base.lo + (int64_t)t * N;
  const uint16_t *eq = J.base.eq + (int64_t)t * N;
  int Kdrop = 0;
  for (int i = 0; i < n_drop; ++i) Kdrop += eq[dlist[i]] > 0;
  const int K = J.base.K[t] - Kdrop;
  long long tie = 0;
  for (int k = lane; k < Np; k += 32) {
    int a = 0;
    if (k < N && eq[k] > 0 && !((dmask[k >> 5] >> (k & 31)) & 1u)) {
      const int lk = lo[k];
      int l = lk, e = eq[k];
      for (int i = 0; i < n_drop; ++i) {
        const int q = dlist[i];
        if (eq[q] > 0) {
          l -= lo[q] < lk;
          e -= lo[q] == lk;
        }
      }
      tie += (long long)e * e - 1;
      a = 2 * l + e - K;
    }
    J.A[(int64_t)t * Np + k] = __int2half_rn(a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tie += __shfl_xor_sync(0xffffffffu, tie, o);
  if (lane == 0) {
    J.tie[t] = tie;
    J.K[t] = K;
  }
}

// The FP64 trait constants of every bucket, one thread per row (FP64 issue is
// slow on this part, so it gets whole warps); padding rows get cfac 0, tau +inf.
__global__ void __launch_bounds__(256) rerank_consts_kernel(const RerankJob *__restrict__ jobs) {
  const RerankJob &J = jobs[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J.rows_pad) return;
  float tau = __int_as_float(0x7f800000);
  double cfac = 0.0;
  if (t < J.T) trait_consts(J.K[t], J.tie[t], tau, cfac);
  J.tau[t] = tau;
  J.cfac[t] = cfac;
}
}  // namespace

cudaError_t launch_rerank_buckets(const RerankJob *jobs, const int32_t *drops, int n_jobs,
                                  int max_rows_pad, cudaStream_t s) {
  for (int j0 = 0; j0 < n_jobs; j0 += 65535) {  // grid.y limit
    const int nj = n_jobs - j0 < 65535 ? n_jobs - j0 : 65535;
    rerank_kernel<<<dim3((unsigned)((max_rows_pad + 7) / 8), (unsigned)nj), 256, 0, s>>>(jobs + j0,
                                                                                       drops);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rerank_consts_kernel<<<dim3((unsigned)((max_rows_pad + 255) / 256), (unsigned)nj), 256, 0, s>>>(
        jobs + j0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace krux
