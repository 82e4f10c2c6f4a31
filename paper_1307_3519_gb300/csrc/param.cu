// param.cu -- parametric comparison statistics on the same tiles (the paper
// compares kruX with matrix-eQTL's linear and ANOVA models on the same data).
//
// The contraction is the one of the Kruskal-Wallis scan with the centred ranks
// replaced by standardised values z = (x - mean) / sd (FP16, so the fused test is
// approximate): with S_i = sum of z over genotype group i,
//   ANOVA:  SS_between = sum_i S_i^2 / N_i (sum_i S_i = 0), compared with the
//           per-df bound tau_df = (K-1) F_c df / (K - 1 - df + F_c df);
//   linear: S_zg = S_1 + 2 S_2 = -(2 S_0 + S_1), compared with the bound
//           S_zg^2 >= r_c^2 S_gg (K - 1), r_c^2 = t_c^2 / (K - 2 + t_c^2).
// Every pair at or above the lower edge of a wide band is kept as a provisional
// hit; this file's finalisation recomputes each one in FP64 from the caller's
// FP32 values, and the filter keeps those with p < P_c.
#include "common.cuh"
#include "param_tails.cuh"

namespace krux {

namespace {

// One warp per trait: FP64 mean and sample standard deviation of the row, the
// standardised FP16 row of A (0 in the padding columns), and the trait constants
// the scan reads (bound 1, no NaN).  A NaN sets kDevBadCode.
__global__ void standardize_kernel(const float *__restrict__ expr, int T, int N, int64_t ld, int Np,
                                   __half *__restrict__ A, double *__restrict__ mean,
                                   double *__restrict__ sd, float *__restrict__ tau,
                                   double *__restrict__ cfac, uint16_t *__restrict__ nan_cnt,
                                   unsigned int *status) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= T) return;
  const float *x = expr + (int64_t)warp * ld;
  double s = 0.0;
  bool nan = false;
  for (int k = lane; k < N; k += 32) {
    const float v = x[k];
    nan |= v != v;
    s += (double)v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double m = s / (double)N;
  double q = 0.0;
  for (int k = lane; k < N; k += 32) {
    const double d = (double)x[k] - m;
    q += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  nan = __any_sync(0xffffffffu, nan);
  const double sdv = N > 1 ? sqrt(q / (double)(N - 1)) : 0.0;
  const double inv = sdv > 0.0 ? 1.0 / sdv : 0.0;
  __half *row = A + (int64_t)warp * Np;
  for (int k = lane; k < Np; k += 32)
    row[k] = __double2half(k < N ? ((double)x[k] - m) * inv : 0.0);
  if (lane == 0) {
    if (nan) atomicOr(status, kDevBadCode);
    mean[warp] = m;
    sd[warp] = sdv;
    // a constant row can never be significant: bound +inf
    tau[warp] = sdv > 0.0 ? 1.0f : __int_as_float(0x7f800000);
    cfac[warp] = 1.0;
    nan_cnt[warp] = 0;
  }
}

// FP64 statistic and p of provisional hit i from the caller's FP32 values.
__global__ void finalize_param_kernel(const krux_hit *__restrict__ hits,
                                      const unsigned long long *__restrict__ count,
                                      int64_t capacity, const float *__restrict__ expr, int64_t ld,
                                      const int8_t *__restrict__ geno, int64_t ldg, int N,
                                      const double *__restrict__ mean, int model,
                                      double *__restrict__ stat, double *__restrict__ P) {
  const unsigned long long c = *count;
  const int64_t n = c < (unsigned long long)capacity ? (int64_t)c : capacity;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const krux_hit r = ld_hit(hits + i);
    const float *x = expr + (int64_t)r.trait * ld;
    const int8_t *g = geno + (int64_t)r.snp * ldg;
    const double m = mean[r.trait];
    double s[3] = {0.0, 0.0, 0.0}, q[3] = {0.0, 0.0, 0.0};
    int cnt[3] = {0, 0, 0};
    for (int k = 0; k < N; ++k) {
      const int code = g[k];
      if (code < 0 || code > 2) continue;
      const double d = (double)x[k] - m;
      s[code] += d;
      q[code] += d * d;
      cnt[code] += 1;
    }
    const int K = cnt[0] + cnt[1] + cnt[2];
    const double st = s[0] + s[1] + s[2];
    double value = 0.0, p = 1.0;
    if (model == 0) {  // one-way ANOVA
      int groups = 0;
      double ssb = 0.0, ssw = 0.0;
      for (int j = 0; j < 3; ++j) {
        if (cnt[j] == 0) continue;
        ++groups;
        ssb += s[j] * s[j] / (double)cnt[j];
        ssw += q[j] - s[j] * s[j] / (double)cnt[j];
      }
      ssb -= st * st / (double)K;
      if (ssw < 0.0) ssw = 0.0;
      if (groups >= 2 && K > groups) {
        const double d1 = groups - 1, d2 = K - groups;
        if (ssw > 0.0) {
          value = (ssb / d1) / (ssw / d2);
          p = f_tail(value, d1, d2);
        } else if (ssb > 0.0) {
          value = __longlong_as_double(0x7ff0000000000000ll);
          p = 0.0;
        }
      }
    } else {  // dosage regression
      const double gs = (double)cnt[1] + 2.0 * cnt[2];
      const double gm = K > 0 ? gs / K : 0.0;
      const double sgg = (double)cnt[1] + 4.0 * cnt[2] - gs * gm;
      const double sxg = s[1] + 2.0 * s[2] - gm * st;
      const double sxx = q[0] + q[1] + q[2] - st * st / (double)K;
      if (K >= 3 && sgg > 0.0 && sxx > 0.0) {
        const double rr = sxg / sqrt(sgg * sxx);
        if (fabs(rr) < 1.0) {
          value = rr * sqrt((K - 2) / (1.0 - rr * rr));
          p = t_tail2(value, (double)(K - 2));
        } else {
          value = rr > 0 ? __longlong_as_double(0x7ff0000000000000ll)
                         : -__longlong_as_double(0x7ff0000000000000ll);
          p = 0.0;
        }
      }
    }
    stat[i] = value;
    P[i] = p;
  }
}

// Keeps the provisional hits with p < P_c: record, statistic and p to the
// caller's lists (d0 = d1 = 0: parametric hits carry no rank sums).
__global__ void filter_param_kernel(const krux_hit *__restrict__ hits,
                                    const unsigned long long *__restrict__ count, int64_t capacity,
                                    const double *__restrict__ stat, const double *__restrict__ P,
                                    double pthresh, krux_hit *__restrict__ out,
                                    double *__restrict__ out_stat, double *__restrict__ out_p,
                                    int64_t out_capacity, unsigned long long *__restrict__ n_out) {
  const unsigned long long c = *count;
  const int64_t n = c < (unsigned long long)capacity ? (int64_t)c : capacity;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!(P[i] < pthresh)) continue;
    const unsigned long long o = atomicAdd(n_out, 1ull);
    if (o < (unsigned long long)out_capacity) {
      krux_hit r = ld_hit(hits + i);
      r.d0 = 0;
      r.d1 = 0;
      st_hit(out + o, r);
      out_stat[o] = stat[i];
      out_p[o] = P[i];
    }
  }
}

}  // namespace

cudaError_t launch_standardize(const float *expr, int T, int N, int64_t ld, int Np, __half *A,
                               double *mean, double *sd, float *tau, double *cfac,
                               uint16_t *nan_cnt, unsigned int *status, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  const int warps_per_block = 8;
  const int grid = (T + warps_per_block - 1) / warps_per_block;
  standardize_kernel<<<grid, warps_per_block * 32, 0, s>>>(expr, T, N, ld, Np, A, mean, sd, tau,
                                                           cfac, nan_cnt, status);
  return cudaGetLastError();
}

cudaError_t launch_finalize_param(const krux_hit *hits, const unsigned long long *count,
                                  int64_t capacity, const float *expr, int64_t ld,
                                  const int8_t *geno, int64_t ldg, int N, const double *mean,
                                  int model, double *stat, double *P, int sm_count,
                                  cudaStream_t s) {
  if (capacity <= 0) return cudaSuccess;
  int grid = sm_count * 4;
  const int64_t need = (capacity + 127) / 128;
  if (need < grid) grid = (int)need;
  finalize_param_kernel<<<grid, 128, 0, s>>>(hits, count, capacity, expr, ld, geno, ldg, N, mean,
                                             model, stat, P);
  return cudaGetLastError();
}

cudaError_t launch_filter_param(const krux_hit *hits, const unsigned long long *count,
                                int64_t capacity, const double *stat, const double *P,
                                double pthresh, krux_hit *out, double *out_stat, double *out_p,
                                int64_t out_capacity, unsigned long long *n_out, int sm_count,
                                cudaStream_t s) {
  if (capacity <= 0) return cudaSuccess;
  int grid = sm_count * 4;
  const int64_t need = (capacity + 255) / 256;
  if (need < grid) grid = (int)need;
  filter_param_kernel<<<grid, 256, 0, s>>>(hits, count, capacity, stat, P, pthresh, out, out_stat,
                                           out_p, out_capacity, n_out);
  return cudaGetLastError();
}

// Host-side thresholds of the fused test.
double param_f_crit(double pthresh, double d1, double d2) {
  double lo = 0.0, hi = 1.0;
  while (f_tail(hi, d1, d2) > pthresh && hi < 1e300) hi *= 2.0;
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (f_tail(mid, d1, d2) > pthresh) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

double param_t_crit(double pthresh, double nu) {
  double lo = 0.0, hi = 1.0;
  while (t_tail2(hi, nu) > pthresh && hi < 1e300) hi *= 2.0;
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (t_tail2(mid, nu) > pthresh) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace krux

// Test hook: the tails above evaluated on the host (no GPU needed).
extern "C" double krux_debug_tail(int kind, double x, double d1, double d2) {
  if (kind == 0) return krux::f_tail(x, d1, d2);
  if (kind == 1) return krux::t_tail2(x, d1);
  return krux::ibeta(d1, d2, x);
}
