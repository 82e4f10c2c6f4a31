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
// With M = K^3 - K - sum(t^3-t) (an exact integer), K(K+1)C = M/(K-1): cfac is one
// correctly rounded FP64 division, 3(K-1)/M, and tau an FP32 one.
__device__ __forceinline__ void trait_consts(int K, long long tie, float &tau, double &cfac) {
  const long long M = K >= 2 ? (long long)K * K * K - K - tie : 0;
  if (M > 0) {
    cfac = 3.0 * (double)(K - 1) / (double)M;
    tau = (float)M / (float)(3 * (K - 1));
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
    // the tile's traits with NaN (low 16 bits) and with more than kNanCMax (high)
    if (N - K > 0) atomicAdd(&r.tile_nan[t / kTileM], 1u + (N - K > kNanCMax ? 1u << 16 : 0u));
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
// eq' = eq - #{q dropped, present, lo_q == lo_k}.
//
// One warp per trait row and kRerankChunk buckets of a run (buckets of one base
// rank set; grid.y = chunk of buckets): the row's lo and eq are read once, into
// registers (lane l owns samples 4l..4l+3 of every 128) and into the warp's
// shared-memory copy (where the dropped samples' values are looked up), the
// chunk's job fields are staged in shared memory, then each bucket costs a pass
// over the registers, one 8-byte store per lane and 128 samples, and an integer
// reduction of the tie sum.  Lane b keeps bucket b's K and tie sum and turns them
// into the FP64 constants at the end, all buckets of the chunk at once.
namespace krux {
namespace {
constexpr int kRerankWarps = 8;
constexpr int kRerankChunk = 16;            // buckets per warp
constexpr int kRerankDrops = 1024;          // drop-list entries staged per block

struct RerankOut {  // a bucket's outputs and drop list, staged per block
  __half *A;
  int64_t *tie;
  int32_t *K;
  float *tau;
  double *cfac;
  int32_t drop_off, n_drop;
};

// kPasses = ceil(Np / 128) passes of 4 samples per lane (the row in registers).
template <int kPasses>
__global__ void __launch_bounds__(kRerankWarps * 32, kPasses == 1 ? 5 : (kPasses == 2 ? 2 : 1))
rerank_kernel(const RerankJob *__restrict__ jobs, int n_jobs_all, const int32_t *__restrict__ drops) {
  __shared__ uint32_t srow[kRerankWarps][kMaxN];  // lo | eq << 16 of the warp's row
  __shared__ RerankOut sj[kRerankChunk];
  __shared__ int32_t sdrop[kRerankDrops];          // the chunk's drop lists, when they fit
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jbase = blockIdx.y * kRerankChunk;
  const int n_jobs = min(kRerankChunk, n_jobs_all - jbase);
  if (threadIdx.x < n_jobs) {
    const RerankJob &J = jobs[jbase + threadIdx.x];
    sj[threadIdx.x] = RerankOut{J.A, J.tie, J.K, J.tau, J.cfac, J.drop_off, J.n_drop};
  }
  __syncthreads();
  // the chunk's drop lists lie back to back in `drops`
  const int d0 = sj[0].drop_off;
  const int nd = sj[n_jobs - 1].drop_off + sj[n_jobs - 1].n_drop - d0;
  const bool staged = nd <= kRerankDrops;
  if (staged)
    for (int i = threadIdx.x; i < nd; i += blockDim.x) sdrop[i] = drops[d0 + i];
  __syncthreads();
  const RerankJob &J0 = jobs[0];  // every job of the run has this base and shape
  const int N = J0.N, Np = J0.Np, T = J0.T, rows_pad = J0.rows_pad;
  const int t = blockIdx.x * kRerankWarps + warp;
  if (t >= rows_pad) return;  // whole warps leave; no block barrier follows
  if (t >= T) {  // padding row: zeros, never a hit
    for (int j = 0; j < n_jobs; ++j) {
      const RerankOut &J = sj[j];
      for (int k = lane; k < Np; k += 32) J.A[(int64_t)t * Np + k] = __int2half_rn(0);
      if (lane == 0) {
        J.tau[t] = __int_as_float(0x7f800000);
        J.cfac[t] = 0.0;
      }
    }
    return;
  }
  const uint16_t *lo = J0.base.lo + (int64_t)t * N;
  const uint16_t *eq = J0.base.eq + (int64_t)t * N;
  for (int k = lane; k < N; k += 32) srow[warp][k] = (uint32_t)lo[k] | ((uint32_t)eq[k] << 16);
  uint32_t own[kPasses][4];
#pragma unroll
  for (int ps = 0; ps < kPasses; ++ps)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 128 * ps + 4 * lane + i;
      own[ps][i] = k < N ? (uint32_t)lo[k] | ((uint32_t)eq[k] << 16) : 0u;
    }
  __syncwarp();
  const int K0 = J0.base.K[t];
  int myK = 0, mytie = 0;  // bucket lane's, for the constants
  for (int j = 0; j < n_jobs; ++j) {
    const RerankOut &J = sj[j];
    const int n_drop = J.n_drop;
    const int32_t *dl = staged ? sdrop + (J.drop_off - d0) : drops + J.drop_off;
    int Kdrop = 0;  // dropped samples with a value
    for (int d = 0; d < n_drop; ++d) Kdrop += (srow[warp][dl[d]] >> 16) > 0u;
    const int K = K0 - Kdrop;
    int tie = 0;
#pragma unroll
    for (int ps = 0; ps < kPasses; ++ps) {
      const int k0 = 128 * ps + 4 * lane;
      int lk[4], l[4], e[4];
      bool present[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        lk[i] = (int)(own[ps][i] & 0xffffu);
        l[i] = lk[i];
        e[i] = (int)(own[ps][i] >> 16);
        present[i] = e[i] > 0;
      }
      for (int d = 0; d < n_drop; ++d) {
        const int q = dl[d];
        const uint32_t w = srow[warp][q];
        const int lq = (int)(w & 0xffffu);
        const bool qp = (w >> 16) > 0u;  // the dropped sample has a value
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          present[i] = present[i] && q != k0 + i;
          l[i] -= qp && lq < lk[i];
          e[i] -= qp && lq == lk[i];
        }
      }
      int a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = 0;
        if (present[i]) {
          tie += e[i] * e[i] - 1;
          a[i] = 2 * l[i] + e[i] - K;
        }
      }
      if (k0 < Np) {
        const __half2 h01 = __halves2half2(__int2half_rn(a[0]), __int2half_rn(a[1]));
        const __half2 h23 = __halves2half2(__int2half_rn(a[2]), __int2half_rn(a[3]));
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t *>(&h01);
        v.y = *reinterpret_cast<const uint32_t *>(&h23);
        *reinterpret_cast<uint2 *>(J.A + (int64_t)t * Np + k0) = v;
      }
    }
    tie = (int)__reduce_add_sync(0xffffffffu, (unsigned)tie);
    if (lane == 0) {
      J.tie[t] = tie;
      J.K[t] = K;
    }
    if (lane == j) {
      myK = K;
      mytie = tie;
    }
  }
  if (lane < n_jobs) {  // the chunk's FP64 constants, one bucket per lane
    float tau;
    double cfac;
    trait_consts(myK, (long long)mytie, tau, cfac);
    sj[lane].tau[t] = tau;
    sj[lane].cfac[t] = cfac;
  }
}
}  // namespace

// One launch per run of buckets with the same base rank set (hjobs: the host copy
// of the device table djobs).
cudaError_t launch_rerank_buckets(const RerankJob *djobs, const RerankJob *hjobs,
                                  const int32_t *drops, int n_jobs, cudaStream_t s) {
  for (int j0 = 0; j0 < n_jobs;) {
    int j1 = j0 + 1;
    while (j1 < n_jobs && hjobs[j1].base.lo == hjobs[j0].base.lo) ++j1;
    const int rows_pad = hjobs[j0].rows_pad;
    const dim3 grid((unsigned)((rows_pad + kRerankWarps - 1) / kRerankWarps),
                    (unsigned)((j1 - j0 + kRerankChunk - 1) / kRerankChunk));
    const int Np = hjobs[j0].Np;
    if (Np <= 128)
      rerank_kernel<1><<<grid, kRerankWarps * 32, 0, s>>>(djobs + j0, j1 - j0, drops);
    else if (Np <= 256)
      rerank_kernel<2><<<grid, kRerankWarps * 32, 0, s>>>(djobs + j0, j1 - j0, drops);
    else
      rerank_kernel<4><<<grid, kRerankWarps * 32, 0, s>>>(djobs + j0, j1 - j0, drops);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    j0 = j1;
  }
  return cudaSuccess;
}
}  // namespace krux
