// plain.cu -- the plain two-pass form of the scan, kept as the measured
// comparison point for the fused kernel: a library FP16 GEMM writes the
// T x (2 * slice) matrix of centred rank sums to device memory (Eq. 4, one SNP
// slice at a time as in section "Data slicing"), then a separate epilogue
// kernel reads it back and evaluates Eq. 2, the tie factor, the chi-square
// threshold and the hit list.
#include <cublas_v2.h>

#include "common.cuh"

namespace krux {

void *plain_handle_create() {
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
  return h;
}

void plain_handle_destroy(void *h) {
  if (h) cublasDestroy(static_cast<cublasHandle_t>(h));
}

// C[t][col] = sum_k A[t][k] * B[col][k]  (row-major C, ldc = rowsB)
cudaError_t plain_gemm(void *handle, const __half *A, int T_rows, int Np, const __half *B, int rowsB,
                       float *C, cudaStream_t s) {
  cublasHandle_t h = static_cast<cublasHandle_t>(handle);
  if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  const float alpha = 1.f, beta = 0.f;
  const cublasStatus_t st =
      cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, rowsB, T_rows, Np, &alpha, B, CUDA_R_16F, Np, A,
                   CUDA_R_16F, Np, &beta, C, CUDA_R_32F, rowsB, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  return st == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

namespace {

__device__ __forceinline__ double p64_of(double H, int df) {
  if (df == 1) return erfc(sqrt(0.5 * H));
  if (df == 2) return exp(-0.5 * H);
  return 1.0;
}

// One thread per (trait, SNP slot of the slice); a warp covers 32 SNPs of one trait.
__global__ void __launch_bounds__(256)
plain_epilogue_kernel(const float *__restrict__ C, int64_t ldc, int T, int n_slots,
                      const ChunkMeta *__restrict__ meta, const float *__restrict__ tau,
                      const double *__restrict__ cfac, const uint16_t *__restrict__ nan_cnt,
                      const uint16_t *__restrict__ nan_idx, int N, const int8_t *__restrict__ geno,
                      int64_t ldg, float margin, double pthresh, float h1, float h2,
                      krux_hit *hits, HitAux *aux, unsigned long long *counter, int64_t capacity,
                      double *dense_H, double *dense_p, int64_t dense_ld, int64_t dense_snp0) {
  const int t = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool hit = false;
  int u = 0, v = 0, n0 = 0, n1 = 0, n2 = 0, snp = -1;
  if (j < n_slots) {
    const int c = j / kChunkSnps, jj = j % kChunkSnps;
    const ChunkMeta &m = meta[c];
    snp = m.snp[jj];
    const float uf = C[(int64_t)t * ldc + (int64_t)c * kChunkRows + jj];
    const float vf = C[(int64_t)t * ldc + (int64_t)c * kChunkRows + kChunkSnps + jj];
    u = (int)uf;
    v = (int)vf;
    n0 = m.n[0][jj];
    n1 = m.n[1][jj];
    n2 = m.n[2][jj];
    const int nn = nan_cnt ? nan_cnt[t] : 0;
    if (snp >= 0 && nn > 0) {
      const int8_t *g = geno + (int64_t)snp * ldg;
      for (int i = 0; i < nn; ++i) {
        const int code = g[nan_idx[(int64_t)t * N + i]];
        n0 -= code == 0;
        n1 -= code == 1;
        n2 -= code == 2;
      }
    }
    const int groups = (n0 > 0) + (n1 > 0) + (n2 > 0);
    const int df = groups > 0 ? groups - 1 : 0;
    const float tf = tau[t];  // K(K+1)C/3, +inf for degenerate traits; 1/tf = 3/(K(K+1)C)
    if (dense_H) {
      if (snp >= 0) {
        const double cf = cfac[t];
        double H = 0.0;
        if (df > 0 && cf > 0.0) {
          const double D0 = u, D1 = v, D2 = -(double)(u + v);
          double Q = 0.0;
          if (n0) Q += D0 * D0 / n0;
          if (n1) Q += D1 * D1 / n1;
          if (n2) Q += D2 * D2 / n2;
          H = cf * Q;
        }
        const double pv = (df > 0 && cf > 0.0) ? p64_of(H, df) : 1.0;
        const int64_t o = (int64_t)t * dense_ld + (snp - dense_snp0);
        dense_H[o] = H;
        dense_p[o] = pv;
        hit = pv < pthresh;
      }
    } else if (snp >= 0 && df > 0 && tf < __int_as_float(0x7f800000)) {
      float hq, hd;
      if (nn == 0) {
        // alpha (u + beta v)^2 + gamma v^2 against tau (1 -/+ margin), as in the fused kernel
        const float w = fmaf(m.beta[jj], vf, uf);
        hq = fmaf(m.alpha[jj] * w, w, m.gamma[jj] * vf * vf);
        hd = tf;
      } else {
        const float w = -(uf + vf);
        float Q = 0.f;
        if (n0) Q += uf * uf / (float)n0;
        if (n1) Q += vf * vf / (float)n1;
        if (n2) Q += w * w / (float)n2;
        hq = Q / tf;
        hd = df == 1 ? h1 : h2;
      }
      if (hq >= hd * (1.f - margin)) {
        hit = hq > hd * (1.f + margin);
        if (!hit) {
          const double D0 = u, D1 = v, D2 = -(double)(u + v);
          double Qd = 0.0;
          if (n0) Qd += D0 * D0 / n0;
          if (n1) Qd += D1 * D1 / n1;
          if (n2) Qd += D2 * D2 / n2;
          hit = p64_of(cfac[t] * Qd, df) < pthresh;
        }
      }
    }
  }
  const unsigned ball = __ballot_sync(0xffffffffu, hit);
  if (ball == 0u) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(counter, (unsigned long long)__popc(ball));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (hit) {
    const unsigned long long idx = base + __popc(ball & ((1u << lane) - 1u));
    if (idx < (unsigned long long)capacity) {
      krux_hit r;
      r.trait = (uint32_t)t;
      r.snp = (uint32_t)snp;
      r.d0 = u;
      r.d1 = v;
      st_hit(hits + idx, r);
      HitAux a;
      a.n0 = (uint16_t)n0;
      a.n1 = (uint16_t)n1;
      a.n2 = (uint16_t)n2;
      a.group = 0;
      st_aux(aux + idx, a);
    }
  }
}

}  // namespace

cudaError_t launch_plain_epilogue2(const float *C, int64_t ldc, int T, int n_slots,
                                   const ChunkMeta *meta, const float *tau, const double *cfac,
                                   const uint16_t *nan_cnt, const uint16_t *nan_idx, int N,
                                   const int8_t *geno, int64_t ldg, float margin, double pthresh,
                                   float h1, float h2, krux_hit *hits, HitAux *aux,
                                   unsigned long long *counter, int64_t capacity, double *dense_H,
                                   double *dense_p, int64_t dense_ld, int64_t dense_snp0,
                                   cudaStream_t s) {
  if (T <= 0 || n_slots <= 0) return cudaSuccess;
  dim3 grid((unsigned)((n_slots + 255) / 256), (unsigned)T);
  plain_epilogue_kernel<<<grid, 256, 0, s>>>(C, ldc, T, n_slots, meta, tau, cfac, nan_cnt, nan_idx,
                                             N, geno, ldg, margin, pthresh, h1, h2, hits, aux,
                                             counter, capacity, dense_H, dense_p, dense_ld,
                                             dense_snp0);
  return cudaGetLastError();
}

}  // namespace krux
