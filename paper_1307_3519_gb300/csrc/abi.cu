// abi.cu -- the C ABI declared in include/krux.h: contexts, rank sets, argument
// validation, device workspace, TMA descriptors, the work schedule of the fused
// scan and the host side of missing-genotype buckets.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace krux;

namespace krux {
cudaError_t launch_missing_scan(const int8_t *geno, int64_t ldg, int N, int64_t snp_begin,
                                int64_t n_snps, int max_code, unsigned int *n_missing,
                                int64_t *miss_idx, uint64_t *miss_mask, unsigned int *status,
                                uint32_t *flags,
                                cudaStream_t s);
cudaError_t launch_pack_linear(const int8_t *geno, int64_t ldg, int N, int Np, int64_t snp_begin,
                               int64_t n_snps, double rl, __half *B, ChunkMeta *meta,
                               unsigned int *status, cudaStream_t s);
cudaError_t launch_standardize(const float *expr, int T, int N, int64_t ld, int Np, __half *A,
                               double *mean, double *sd, float *tau, double *cfac,
                               uint16_t *nan_cnt, unsigned int *status, cudaStream_t s);
cudaError_t launch_finalize_param(const krux_hit *hits, const unsigned long long *count,
                                  int64_t capacity, const float *expr, int64_t ld,
                                  const int8_t *geno, int64_t ldg, int N, const double *mean,
                                  int model, double *stat, double *P, int sm_count,
                                  cudaStream_t s);
cudaError_t launch_filter_param(const krux_hit *hits, const unsigned long long *count,
                                int64_t capacity, const double *stat, const double *P,
                                double pthresh, krux_hit *out, double *out_stat, double *out_p,
                                int64_t out_capacity, unsigned long long *n_out, int sm_count,
                                cudaStream_t s);
double param_f_crit(double pthresh, double d1, double d2);
double param_t_crit(double pthresh, double nu);
cudaError_t launch_pack_multi(const int8_t *geno, int64_t ldg, int N, int Np,
                              const int64_t *snp_list, int64_t snp_begin, int64_t n_snps,
                              const double *h, int allow_missing, __half *B, ChunkMetaM *meta,
                              unsigned int *status, cudaStream_t s);
cudaError_t launch_pack2(const int8_t *geno, int64_t ldg, int N, int Np, const int64_t *snp_list,
                         int64_t snp_begin, int64_t n_snps, int64_t snp_out_base, double h1,
                         double h2, int allow_missing, int signed_df1, __half *B,
                         ChunkMeta *meta, uint64_t *codes, unsigned int *status, cudaStream_t s);
cudaError_t launch_pack_batch(const PackJob *jobs, int n_jobs, int64_t total_slots,
                              int64_t total_halves, double h1, double h2, int signed_df1,
                              unsigned int *status, cudaStream_t s);
cudaError_t launch_rerank_buckets(const RerankJob *djobs, const RerankJob *hjobs,
                                  const int32_t *drops, int n_jobs, cudaStream_t s);
cudaError_t launch_plain_epilogue2(const float *C, int64_t ldc, int T, int n_slots,
                                   const ChunkMeta *meta, const float *tau, const double *cfac,
                                   const uint16_t *nan_cnt, const uint16_t *nan_idx, int N,
                                   const int8_t *geno, int64_t ldg, float margin, double pthresh,
                                   float h1, float h2, krux_hit *hits, HitAux *aux,
                                   unsigned long long *counter, int64_t capacity, double *dense_H,
                                   double *dense_p, int64_t dense_ld, int64_t dense_snp0,
                                   cudaStream_t s);
cudaError_t plain_gemm(void *handle, const __half *A, int T, int Np, const __half *B, int rowsB,
                       float *C, cudaStream_t s);
void *plain_handle_create();
void plain_handle_destroy(void *h);
}  // namespace krux

namespace {

// Pinned host staging buffer (grow-only): uploads from it run at the link's rate.
// A call overwrites it only after the previous call's copies have completed
// (every call synchronises its stream before returning).
struct HostBuf {
  void *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    const size_t want = bytes + bytes / 4 + 4096;
    cudaError_t e = cudaHostAlloc(&p, want, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
  }
};

struct DevBuf {
  void *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    size_t want = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    n = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  template <class T>
  T *as() const {
    return reinterpret_cast<T *>(p);
  }
};

constexpr int kEv = 8;
constexpr long long kDefaultWait = 4000000000LL;  // SM cycles, about two seconds

// chi-square upper-tail thresholds at p for 1 and 2 degrees of freedom:
// P(chi2_1 > h) = erfc(sqrt(h/2)) and P(chi2_2 > h) = exp(-h/2).
double h_df1(double p) {
  // solve erfc(x) = p for x by bisection on a bracketing interval, then Newton
  double lo = 0.0, hi = 40.0;
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (std::erfc(mid) > p) lo = mid; else hi = mid;
  }
  double x = 0.5 * (lo + hi);
  for (int i = 0; i < 3; ++i) {
    const double f = std::erfc(x) - p;
    const double d = -2.0 / std::sqrt(M_PI) * std::exp(-x * x);
    if (d == 0.0) break;
    x -= f / d;
  }
  return 2.0 * x * x;
}
double h_df2(double p) { return -2.0 * std::log(p); }

// Upper chi-square tail for df = 1..4 from the closed forms of Q(df/2, h/2).
double chi2_tail_host(double h, int df) {
  const double x = 0.5 * h;
  if (!(x > 0.0)) return 1.0;
  switch (df) {
    case 1: return std::erfc(std::sqrt(x));
    case 2: return std::exp(-x);
    case 3: return std::erfc(std::sqrt(x)) + 2.0 * std::sqrt(x / M_PI) * std::exp(-x);
    default: return std::exp(-x) * (1.0 + x);
  }
}

// Threshold h_d with P(chi2_d > h_d) = p, d = 1..4 (d = 1, 2 in closed form).
double h_dfk(double p, int df) {
  if (df == 1) return h_df1(p);
  if (df == 2) return h_df2(p);
  double lo = 0.0, hi = 4000.0;  // the tail is decreasing in h
  for (int i = 0; i < 300; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (chi2_tail_host(mid, df) > p) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

struct krux_rankset {
  int T = 0, N = 0, Np = 0, rows_pad = 0, n_ttiles = 0;
  bool has_nan = false;  // decided on the host after ranking
  int nan_traits_over = 0;  // traits with more than kNanCMax NaN samples
  RankDev dev{};
  void *mem = nullptr;
  size_t bytes = 0;
};

struct krux_ctx {
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  std::string err;
  bool profiling = false;
  krux_profile prof{};
  long long wait_limit = kDefaultWait;
  int tune_layout = -1, tune_nc = 0, tune_nA = 0, tune_ka = 0;  // 0 / -1 = automatic
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  cudaEvent_t ev[kEv] = {};
  // krux_scan_host: the genotypes' copy runs on its own stream beside the rank transform
  cudaStream_t xs = nullptr;
  cudaEvent_t xev = nullptr;
  DevBuf B, meta, codes, groups, items, status, counters, aux, cfacptr, miss_idx, miss_mask,
      list, gemm_out, bucket_ranks, permA, minpkey, seg, permNan, aux2, param, paramOut, packjobs,
      host_in, host_out,  // krux_scan_host: device copies of the inputs, device hit list
      groups2, items2, packjobs2, cfacptr2,  // launch tables of a second launch in the same call
      mcand,  // plain-form permutation batches: pairs for the deferred FP64 pass
      pattern, dlist;  // device-side missing-pattern grouping: scratch, SNP lists
  HostBuf list_host;  // staging of the SNP lists
  void *blas = nullptr;
  std::vector<std::pair<size_t, void *>> pool;  // freed rank-set blocks, reused by size
  std::map<int, std::array<int, 4>> tuned;       // krux_autotune: K width -> layout, nc, nA, ka
};

namespace {

krux_status fail(krux_ctx *ctx, krux_status st, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

#define KRUX_CUDA(ctx, call)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? KRUX_ENOMEM : KRUX_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                         \
  } while (0)

int round_up(int x, int m) { return (x + m - 1) / m * m; }

void ev_record(krux_ctx *ctx, int i, cudaStream_t s) {
  if (ctx->profiling) cudaEventRecord(ctx->ev[i], s);
}
float ev_ms(krux_ctx *ctx, int a, int b) {
  float ms = 0.f;
  if (ctx->profiling && cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) == cudaSuccess) return ms;
  return 0.f;
}

int layout_atom(int layout) { return layout ? 16 : kAtomK; }

krux_status encode_map(krux_ctx *ctx, CUtensorMap *map, const void *base, int Np, int64_t rows,
                       int layout) {
  cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Np * 2};
  cuuint32_t box[2] = {(cuuint32_t)layout_atom(layout), (cuuint32_t)kTileM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           layout ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, KRUX_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KRUX_OK;
}

// Pipeline shape of one launch.  The A (rank) stages hold ka samples of 128
// traits: the whole K when that leaves room for at least three resident SNP
// chunks of the widest group, else K blocks of 64 samples.  b_region is the
// shared memory left for resident B chunks; each group keeps as many of its own
// chunks as fit (at most the 4 TMEM accumulator slots, at most 2 when its K is
// split into blocks, so that its accumulators stay double-buffered).
struct LaunchShape {
  int ka = 0, nA = 0, b_region = 0, force_nc = 0, no_pair = 0;
};
constexpr size_t kSmemLimit = 232448;

size_t shape_overhead(int nA, int codes_k) {
  return scan_smem_bytes2(kTmemSlots, nA, 0, 0, std::max(codes_k, 16));
}

// reserve: shared memory kept free for the plain form's hit-event ring (0 when
// the call cannot take that form).
bool pick_launch_shape(const krux_ctx *ctx, int kpad, int codes_k, LaunchShape &sh,
                       size_t reserve = 0) {
  const size_t chunk = (size_t)256 * kpad;
  if (ctx->tune_nc > 0) {  // explicit shape (tests, autotuner)
    sh.ka = ctx->tune_ka > 0 ? ctx->tune_ka : kpad;
    sh.nA = ctx->tune_nA;
    sh.b_region = (int)(chunk * ctx->tune_nc);
    sh.force_nc = ctx->tune_nc;
    if (sh.ka % 64 != 0 && sh.ka != kpad) return false;
    return shape_overhead(sh.nA, codes_k) + (size_t)sh.nA * 256 * sh.ka + sh.b_region <= kSmemLimit;
  }
  if (reserve > 0) {  // the plain form: whole K per stage and an even number of chunks
    int best = 0;
    for (int a = 3; a >= 2; --a) {
      const size_t used = shape_overhead(a, codes_k) + (size_t)a * chunk + reserve;
      if (used >= kSmemLimit) continue;
      const int ncf = (int)std::min<size_t>(kTmemSlots, (kSmemLimit - used) / chunk) & ~1;
      if (ncf > best) {
        best = ncf;
        sh.ka = kpad;
        sh.nA = a;
        sh.b_region = (int)(ncf * chunk);
      }
    }
    if (best >= 2) return true;
  }
  for (int a = 3; a >= 2; --a) {  // whole K per stage
    const size_t used = shape_overhead(a, codes_k) + (size_t)a * chunk;
    if (used < kSmemLimit && (kSmemLimit - used) / chunk >= 3) {
      sh.ka = kpad;
      sh.nA = a;
      sh.b_region = (int)(std::min<size_t>(kTmemSlots, (kSmemLimit - used) / chunk) * chunk);
      return true;
    }
  }
  int best_nc = 0;
  for (int a = 4; a >= 2; --a) {  // K blocks of 64 samples
    const size_t used = shape_overhead(a, codes_k) + (size_t)a * 256 * 64;
    if (used >= kSmemLimit) continue;
    // keep every region after B on a 1024-byte boundary (TMA and vector loads)
    const size_t region = (kSmemLimit - used) / 1024 * 1024;
    const int nc = (int)std::min<size_t>(2, region / chunk);
    if (nc > best_nc) {
      best_nc = nc;
      sh.ka = 64;
      sh.nA = a;
      sh.b_region = (int)region;
    }
  }
  return best_nc >= 1;
}

// True when a group of this width can take the plain scan form: a launch shape
// with the whole K per rank stage, an even number of resident chunks and room for
// the hit-event ring (the 32-byte swizzle layout).
bool plain_form_fits(const krux_ctx *ctx, int Np) {
  if (ctx->tune_layout == 0) return false;
  const int kpad = round_up(Np, 16);
  LaunchShape sh;
  if (!pick_launch_shape(ctx, kpad, 0, sh, kEvRegion)) return false;
  const int nc = (int)(sh.b_region / (256 * kpad));
  return sh.ka == kpad && nc >= 2 && nc % 2 == 0 &&
         shape_overhead(sh.nA, 0) + (size_t)sh.nA * 256 * sh.ka + sh.b_region + kEvRegion <= kSmemLimit;
}

// Refuses a launch plan whose shared-memory regions or per-group shapes are not
// aligned or do not fit: every TMA destination and vector load must stay
// aligned and inside its region.  Returns an empty string when the plan is sound.
std::string validate_plan(const ScanParams &p, const std::vector<GroupDesc> &g, size_t smem) {
  char buf[256];
  auto bad = [&](const char *what) {
    snprintf(buf, sizeof buf, "internal launch plan check failed: %s", what);
    return std::string(buf);
  };
  const int atom = p.layout ? 16 : 64;
  if (smem > kSmemLimit) return bad("shared memory above the per-CTA limit");
  if (p.nA < 1 || p.nc < 1 || p.nc > kTmemSlots) return bad("stage or chunk count");
  if (p.a_tile_bytes % 1024 || p.b_region % 1024 || p.a_tile_bytes != 256 * p.ka) return bad("region alignment");
  if (p.ka % atom || p.kpad < 16) return bad("K widths");
  if ((size_t)p.nA * p.a_tile_bytes + (size_t)p.b_region + 1024 > smem) return bad("regions exceed the allocation");
  for (const GroupDesc &d : g) {
    if (d.nc < 1 || d.nc > p.nc) return bad("group chunk count");
    if (d.b_stride % 4096 || (int64_t)d.nc * d.b_stride > p.b_region) return bad("group B chunks");
    if (d.b_stride < 256 * d.n_atoms * atom) return bad("group B stride");
    if ((int64_t)d.nkb * p.ka < (int64_t)d.n_atoms * atom || d.nkb < 1) return bad("group K blocks");
    if (d.nkb > 1 && d.nc * 2 > kTmemSlots) return bad("TMEM slots for K blocks");
    if (d.Np % 16 || d.Np > d.n_atoms * atom) return bad("group K width");
    if (d.codes && (d.codes_k > p.kpad || d.codes_k < 1)) return bad("codes width");
    if (d.pair && (p.layout != 1 || d.nc % 2 != 0)) return bad("chunk pairs");
  }
  return std::string();
}

// Per-group share of a launch shape.
void group_shape(const LaunchShape &sh, int kpad_g, int atom, GroupDesc &d) {
  d.b_stride = 256 * kpad_g;
  const int atoms_per_block = sh.ka / atom;
  d.nkb = (d.n_atoms + atoms_per_block - 1) / atoms_per_block;
  int nc = (int)std::min<int64_t>(kTmemSlots, sh.b_region / d.b_stride);
  if (d.nkb > 1) nc = std::min(nc, 2);
  if (sh.force_nc > 0) nc = std::min(nc, sh.force_nc);
  d.nc = std::max(nc, 1);
  // N = 256 MMAs over chunk pairs (32-byte swizzle layout, even chunk count)
  d.pair = (atom == 16 && d.nc >= 2 && d.nc % 2 == 0 && !sh.no_pair) ? 1 : 0;
}

struct GroupPlan {
  GroupDesc d;
  int64_t n_btiles = 0;
  int64_t steps = 0;
  int64_t step_lo = 0;  // first step scanned (a min-p seed pass skips the unpermuted agroup)
};

std::vector<WorkItem> make_items(const std::vector<GroupPlan> &gp, int nc, int grid) {
  int64_t nb = 0, maxL = 1;
  for (auto &g : gp) {
    nb += g.n_btiles;
    maxL = std::max(maxL, g.steps - g.step_lo);
  }
  int best_split = 1;
  double best = 1e300;
  for (int s = 1; s <= 32 && s <= maxL; ++s) {
    const int64_t items = nb * s;
    const int64_t waves = (items + grid - 1) / grid;
    const double cost = (double)waves * ((double)maxL / s + 2.0);
    if (cost < best * 0.999) {
      best = cost;
      best_split = s;
    }
  }
  std::vector<WorkItem> items;
  for (size_t gi = 0; gi < gp.size(); ++gi) {
    const auto &g = gp[gi];
    const int64_t L = g.steps - g.step_lo;
    const int s = (int)std::min<int64_t>(best_split, L);
    for (int64_t b = 0; b < g.n_btiles; ++b)
      for (int k = 0; k < s; ++k) {
        WorkItem w;
        w.group = (int32_t)gi;
        w.btile = (int32_t)b;
        w.step_begin = (int32_t)(g.step_lo + L * k / s);
        w.step_end = (int32_t)(g.step_lo + L * (k + 1) / s);
        if (w.step_end > w.step_begin) items.push_back(w);
      }
  }
  (void)nc;
  return items;
}

__global__ void export_kernel(const __half *A, int T, int N, int Np, int16_t *out) {
  const int64_t total = (int64_t)T * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i / N;
    const int k = (int)(i % N);
    out[i] = (int16_t)__half2int_rn(A[t * Np + k]);
  }
}

// ranked-set allocation: one cudaMalloc carved into the RankDev arrays
krux_status alloc_rankset(krux_ctx *ctx, krux_rankset *rs, int T, int N, bool with_lists) {
  rs->T = T;
  rs->N = N;
  rs->Np = round_up(N, 16);
  rs->rows_pad = round_up(std::max(T, 1), kTileM);
  rs->n_ttiles = rs->rows_pad / kTileM;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t oA = take((size_t)rs->rows_pad * rs->Np * 2);
  const size_t olo = with_lists ? take((size_t)T * N * 2) : 0;
  const size_t oeq = with_lists ? take((size_t)T * N * 2) : 0;
  const size_t otie = take((size_t)T * 8);
  const size_t oK = take((size_t)T * 4);
  const size_t otau = take((size_t)rs->rows_pad * 4);
  const size_t ocf = take((size_t)rs->rows_pad * 8);
  const size_t onc = take((size_t)rs->rows_pad * 2);
  const size_t oni = take((size_t)T * N * 2);
  const size_t otn = take((size_t)rs->n_ttiles * 4);
  rs->mem = nullptr;
  for (size_t i = 0; i < ctx->pool.size(); ++i) {
    if (ctx->pool[i].first == off) {
      rs->mem = ctx->pool[i].second;
      ctx->pool.erase(ctx->pool.begin() + (long)i);
      break;
    }
  }
  if (!rs->mem) KRUX_CUDA(ctx, cudaMalloc(&rs->mem, off));
  rs->bytes = off;
  char *b = (char *)rs->mem;
  rs->dev.A = (__half *)(b + oA);
  rs->dev.lo = with_lists ? (uint16_t *)(b + olo) : nullptr;
  rs->dev.eq = with_lists ? (uint16_t *)(b + oeq) : nullptr;
  rs->dev.tie = (int64_t *)(b + otie);
  rs->dev.K = (int32_t *)(b + oK);
  rs->dev.tau = (float *)(b + otau);
  rs->dev.cfac = (double *)(b + ocf);
  rs->dev.nan_cnt = (uint16_t *)(b + onc);
  rs->dev.nan_idx = (uint16_t *)(b + oni);
  rs->dev.tile_nan = (uint32_t *)(b + otn);
  return KRUX_OK;
}

krux_status check_opts(krux_ctx *ctx, const krux_opts *o) {
  if (!o) return fail(ctx, KRUX_EINVAL, "opts is NULL");
  if (!(o->pthresh > 0.0 && o->pthresh < 1.0)) return fail(ctx, KRUX_EINVAL, "pthresh must be in (0,1)");
  if (o->hit_capacity < 0) return fail(ctx, KRUX_EINVAL, "hit_capacity < 0");
  if ((o->flags & ~KRUX_FLAG_MULTIALLELIC) != 0) return fail(ctx, KRUX_EINVAL, "unknown flags");
  if ((o->flags & KRUX_FLAG_MULTIALLELIC) && o->dense_H)
    return fail(ctx, KRUX_EINVAL, "dense output is not available for markers with codes 0..4");
  if ((o->dense_H == nullptr) != (o->dense_p == nullptr))
    return fail(ctx, KRUX_EINVAL, "dense_H and dense_p must both be set or both NULL");
  return KRUX_OK;
}

}  // namespace

// ------------------------------------------------------------------------------
extern "C" {

const char *krux_status_string(krux_status s) {
  switch (s) {
    case KRUX_OK: return "ok";
    case KRUX_EINVAL: return "invalid argument";
    case KRUX_ENOMEM: return "out of memory";
    case KRUX_ECUDA: return "CUDA error";
    case KRUX_EOVERFLOW: return "hit list overflow";
    case KRUX_ETIMEOUT: return "device wait timed out";
    case KRUX_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *krux_last_error(const krux_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

krux_status krux_create(krux_ctx **out, int device) {
  if (!out) return KRUX_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return KRUX_EINVAL;
  krux_ctx *ctx = new krux_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return KRUX_ECUDA;
  }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&ctx->cc_major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&ctx->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
  if (!(ctx->cc_major == 10 && ctx->cc_minor == 3)) {
    delete ctx;
    return KRUX_EUNSUPPORTED;
  }
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      fn == nullptr) {
    delete ctx;
    return KRUX_ECUDA;
  }
  ctx->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  for (int i = 0; i < kEv; ++i) cudaEventCreate(&ctx->ev[i]);
  *out = ctx;
  return KRUX_OK;
}

void krux_destroy(krux_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  DevBuf *bufs[] = {&ctx->B, &ctx->meta, &ctx->codes, &ctx->groups, &ctx->items, &ctx->status,
                    &ctx->counters, &ctx->aux, &ctx->cfacptr, &ctx->miss_idx, &ctx->miss_mask,
                    &ctx->list, &ctx->gemm_out, &ctx->bucket_ranks, &ctx->permA, &ctx->minpkey, &ctx->seg,
                    &ctx->permNan, &ctx->aux2, &ctx->param, &ctx->paramOut, &ctx->packjobs,
                    &ctx->host_in, &ctx->host_out, &ctx->groups2, &ctx->items2, &ctx->packjobs2,
                    &ctx->cfacptr2, &ctx->mcand, &ctx->pattern, &ctx->dlist};
  for (DevBuf *b : bufs) b->release();
  ctx->list_host.release();
  for (auto &pb : ctx->pool) cudaFree(pb.second);
  for (int i = 0; i < kEv; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->xev) cudaEventDestroy(ctx->xev);
  if (ctx->xs) cudaStreamDestroy(ctx->xs);
  if (ctx->blas) plain_handle_destroy(ctx->blas);
  delete ctx;
}

krux_status krux_set_profiling(krux_ctx *ctx, int enable) {
  if (!ctx) return KRUX_EINVAL;
  ctx->profiling = enable != 0;
  return KRUX_OK;
}

krux_status krux_get_profile(const krux_ctx *ctx, krux_profile *out) {
  if (!ctx || !out) return KRUX_EINVAL;
  *out = ctx->prof;
  return KRUX_OK;
}

krux_status krux_set_tuning(krux_ctx *ctx, int layout, int nc, int nA, int ka) {
  if (!ctx || layout < -1 || layout > 1 || nc < 0 || nA < 0 || nc > kTmemSlots || nA > 8 ||
      ((nc == 0) != (nA == 0)) || ka < 0 || ka % 64 != 0 || (ka > 0 && nc == 0))
    return KRUX_EINVAL;
  ctx->tune_layout = layout;
  ctx->tune_nc = nc;
  ctx->tune_nA = nA;
  ctx->tune_ka = ka;
  return KRUX_OK;
}

krux_status krux_set_wait_limit(krux_ctx *ctx, long long cycles) {
  if (!ctx || cycles < 0) return KRUX_EINVAL;
  ctx->wait_limit = cycles == 0 ? kDefaultWait : cycles;
  return KRUX_OK;
}

krux_status krux_make_perms(uint64_t seed, int P, int N, int32_t *out) {
  if (P < 0 || N < 0 || (P > 0 && N > 0 && !out)) return KRUX_EINVAL;
  for (int q = 0; q < P; ++q) {
    int32_t *pm = out + (int64_t)q * N;
    for (int k = 0; k < N; ++k) pm[k] = k;
    uint64_t s = seed + (uint64_t)q;
    for (int i = N - 1; i >= 1; --i) {
      s += 0x9E3779B97F4A7C15ull;
      uint64_t z = s;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const int j = (int)(z % (uint64_t)(i + 1));
      std::swap(pm[i], pm[j]);
    }
  }
  return KRUX_OK;
}

krux_status krux_rank(krux_ctx *ctx, const float *expr, int T, int N, int64_t ld,
                      krux_rankset **out, void *stream) {
  if (!ctx || !out) return fail(ctx, KRUX_EINVAL, "NULL argument");
  *out = nullptr;
  if (T < 1 || N < 1 || N > kMaxN || ld < N || !expr)
    return fail(ctx, KRUX_EINVAL, "krux_rank: need T >= 1, 1 <= N <= %d, ld >= N, expr != NULL", kMaxN);
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  krux_rankset *rs = new krux_rankset();
  krux_status st = alloc_rankset(ctx, rs, T, N, true);
  if (st != KRUX_OK) {
    delete rs;
    return st;
  }
  ev_record(ctx, 0, s);
  cudaError_t e = cudaMemsetAsync(rs->dev.A, 0, (size_t)rs->rows_pad * rs->Np * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(rs->dev.tile_nan, 0, (size_t)rs->n_ttiles * 4, s);
  if (e == cudaSuccess) e = launch_rank(expr, T, N, ld, rs->Np, rs->rows_pad, rs->dev, s);
  ev_record(ctx, 1, s);
  uint32_t any_nan = 0;
  if (e == cudaSuccess) {
    std::vector<uint32_t> tn(rs->n_ttiles);
    e = cudaMemcpyAsync(tn.data(), rs->dev.tile_nan, tn.size() * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (uint32_t v : tn) {
      any_nan |= v & 0xffffu;
      rs->nan_traits_over += (int)(v >> 16);
    }
  }
  if (e != cudaSuccess) {
    krux_rankset_free(ctx, rs);
    return fail(ctx, KRUX_ECUDA, "krux_rank: %s", cudaGetErrorString(e));
  }
  rs->has_nan = any_nan != 0;
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    ctx->prof.ms_rank = ev_ms(ctx, 0, 1);
    ctx->prof.launches = 2;  // the rank transform and the padding-row constants
  }
  *out = rs;
  return KRUX_OK;
}

void krux_rankset_free(krux_ctx *ctx, krux_rankset *rs) {
  if (!rs) return;
  if (ctx && rs->mem) {
    ctx->pool.emplace_back(rs->bytes, rs->mem);  // kept for the next krux_rank of this size
  } else if (rs->mem) {
    cudaFree(rs->mem);
  }
  delete rs;
}

krux_status krux_rankset_export(krux_ctx *ctx, const krux_rankset *rs, int16_t *centred,
                                int64_t *tie, int32_t *K, void *stream) {
  if (!ctx || !rs) return fail(ctx, KRUX_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (centred) {
    export_kernel<<<std::max(1, std::min(4096, (rs->T * rs->N + 255) / 256)), 256, 0, s>>>(
        rs->dev.A, rs->T, rs->N, rs->Np, centred);
    KRUX_CUDA(ctx, cudaGetLastError());
  }
  if (tie) KRUX_CUDA(ctx, cudaMemcpyAsync(tie, rs->dev.tie, (size_t)rs->T * 8, cudaMemcpyDeviceToDevice, s));
  if (K) KRUX_CUDA(ctx, cudaMemcpyAsync(K, rs->dev.K, (size_t)rs->T * 4, cudaMemcpyDeviceToDevice, s));
  return KRUX_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------
// Missing genotypes (section "Handling missing values": one genotype matrix per
// missing-value pattern, with the expression re-ranked without those samples).
namespace {

struct Bucket {
  std::vector<int32_t> drop;   // samples removed
  std::vector<int64_t> snps;   // SNP rows with exactly this pattern, ascending (host grouping)
  int64_t dev_off = -1;        // device grouping: the rows at ctx->dlist + dev_off
  int64_t count = 0;           //   (count of them)
};

// Device grouping result: where a call's lists sit in ctx->dlist.
struct DevLists {
  int64_t base = -1;           // first entry this grouping may use (-1: group on the host)
  int64_t complete_off = -1;   // the complete rows at ctx->dlist + complete_off
  int64_t complete_count = 0;
};

// Device-side grouping of the flagged SNPs (after the missing-code pre-pass): the
// buckets' rows and the complete rows are written into ctx->dlist from dl.base on;
// the host reads only the bucket count, sizes, first rows and masks.  Returns false
// (and leaves the host to group) on a hash collision between two patterns.
krux_status group_on_device(krux_ctx *ctx, int N, int64_t b, int64_t n, int64_t m,
                            bool flags_ready, cudaStream_t s, std::vector<Bucket> &buckets,
                            DevLists &dl, bool &done) {
  done = false;
  constexpr int W = kMaxN / 64;
  int64_t cap = 16;
  while (cap < 2 * n) cap <<= 1;
  // scratch layout, each part 256-byte aligned
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_hash = take((size_t)cap * 8), o_rep = take((size_t)cap * 4), o_id = take((size_t)cap * 4);
  const size_t o_slot = take((size_t)n * 4), o_bof = take((size_t)n * 4), o_nb = take(4);
  const size_t o_cnt = take((size_t)n * 4), o_fill = take((size_t)n * 4), o_first = take((size_t)n * 8);
  const size_t o_mask = take((size_t)n * W * 8), o_off = take((size_t)n * 8);
  const size_t o_woff = take((size_t)((n + 31) / 32 + 1) * 8);
  KRUX_CUDA(ctx, ctx->pattern.ensure(off));
  char *pb = ctx->pattern.as<char>();
  PatternScratch w;
  w.tab_hash = reinterpret_cast<unsigned long long *>(pb + o_hash);
  w.tab_rep = reinterpret_cast<int *>(pb + o_rep);
  w.tab_id = reinterpret_cast<int *>(pb + o_id);
  w.slot_of = reinterpret_cast<int *>(pb + o_slot);
  w.bucket_of = reinterpret_cast<int *>(pb + o_bof);
  w.n_buckets = reinterpret_cast<unsigned int *>(pb + o_nb);
  w.count = reinterpret_cast<unsigned int *>(pb + o_cnt);
  w.fill = reinterpret_cast<unsigned int *>(pb + o_fill);
  w.first = reinterpret_cast<unsigned long long *>(pb + o_first);
  w.bucket_mask = reinterpret_cast<uint64_t *>(pb + o_mask);
  w.offset = reinterpret_cast<int64_t *>(pb + o_off);
  w.woff = reinterpret_cast<int64_t *>(pb + o_woff);
  w.cap = cap;
  unsigned int *cnt = ctx->counters.as<unsigned int>();
  unsigned int *status = ctx->status.as<unsigned int>();
  const size_t mask_bytes = (size_t)std::max<int64_t>(n, 1) * (kMaxN / 8);
  uint32_t *flags = reinterpret_cast<uint32_t *>(ctx->miss_mask.as<char>() + mask_bytes);
  KRUX_CUDA(ctx, launch_pattern_group(cnt, ctx->miss_mask.as<uint64_t>(), ctx->miss_idx.as<int64_t>(),
                                      n, w, status, s));
  unsigned int nb = 0, st = 0;
  KRUX_CUDA(ctx, cudaMemcpyAsync(&nb, w.n_buckets, 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  if (st & kDevHashCollision) {
    KRUX_CUDA(ctx, cudaMemsetAsync(status, 0, 64, s));  // the host groups instead
    return KRUX_OK;
  }
  std::vector<unsigned int> count(nb);
  std::vector<unsigned long long> first(nb);
  std::vector<uint64_t> bmask((size_t)nb * W);
  KRUX_CUDA(ctx, cudaMemcpyAsync(count.data(), w.count, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(first.data(), w.first, (size_t)nb * 8, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(bmask.data(), w.bucket_mask, bmask.size() * 8, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  // buckets in order of their first SNP; lists back to back, then the complete rows
  std::vector<int> order(nb);
  for (unsigned int i = 0; i < nb; ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return first[x] < first[y]; });
  std::vector<int64_t> offset(nb);
  int64_t run = 0;
  for (int id : order) {
    offset[id] = run;
    run += count[id];
  }
  KRUX_CUDA(ctx, cudaMemcpyAsync(w.offset, offset.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, s));
  int64_t *lists = ctx->dlist.as<int64_t>() + dl.base;
  KRUX_CUDA(ctx, launch_pattern_lists(cnt, ctx->miss_idx.as<int64_t>(), flags, flags_ready, b, n, w,
                                      lists, lists + m, s));
  buckets.clear();
  for (int id : order) {
    Bucket bk;
    const uint64_t *key = bmask.data() + (size_t)id * W;
    for (int k = 0; k < N; ++k)
      if ((key[k / 64] >> (k % 64)) & 1ull) bk.drop.push_back(k);
    bk.dev_off = dl.base + offset[id];
    bk.count = count[id];
    buckets.push_back(std::move(bk));
  }
  dl.complete_off = dl.base + m;
  dl.complete_count = n - m;
  done = true;
  return KRUX_OK;
}

// Finds SNPs of rows [b, b+n) that carry a -1, groups them by their exact
// missing-sample set, and lists the complete rows.  `bad` reports codes outside
// {-1,0,1,2}.  Synchronises the stream.
krux_status find_missing(krux_ctx *ctx, const int8_t *geno, int64_t ldg, int N, int64_t b,
                         int64_t n, cudaStream_t s, std::vector<Bucket> &buckets,
                         std::vector<int64_t> &complete, bool &bad, int max_code,
                         DevLists *dl = nullptr) {
  KRUX_CUDA(ctx, ctx->status.ensure(64));
  KRUX_CUDA(ctx, ctx->counters.ensure(64));
  KRUX_CUDA(ctx, ctx->miss_idx.ensure((size_t)std::max<int64_t>(n, 1) * 8));
  // the masks, then one flag bit per SNP for the flat pre-pass
  const size_t mask_bytes = (size_t)std::max<int64_t>(n, 1) * (kMaxN / 8);
  KRUX_CUDA(ctx, ctx->miss_mask.ensure(mask_bytes + (size_t)(n + 31) / 32 * 4 + 256));
  KRUX_CUDA(ctx, cudaMemsetAsync(ctx->status.p, 0, 64, s));
  KRUX_CUDA(ctx, cudaMemsetAsync(ctx->counters.p, 0, 64, s));
  unsigned int *cnt = ctx->counters.as<unsigned int>();
  uint32_t *flags = reinterpret_cast<uint32_t *>(ctx->miss_mask.as<char>() + mask_bytes);
  KRUX_CUDA(ctx, launch_missing_scan(geno, ldg, N, b, n, max_code, cnt, ctx->miss_idx.as<int64_t>(),
                                     ctx->miss_mask.as<uint64_t>(), ctx->status.as<unsigned int>(),
                                     flags, s));
  if (ctx->profiling) ctx->prof.launches += ldg == N ? 2 : 1;
  unsigned int m32 = 0, st = 0;
  KRUX_CUDA(ctx, cudaMemcpyAsync(&m32, cnt, 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(&st, ctx->status.p, 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  bad = (st & kDevBadCode) != 0;
  buckets.clear();
  complete.clear();
  if (bad || m32 == 0) return KRUX_OK;
  const int64_t m = m32;
  if (dl && dl->base >= 0) {  // group on the device when the lists have room there
    bool done = false;
    krux_status gs = group_on_device(ctx, N, b, n, m, ldg == N, s, buckets, *dl, done);
    if (gs != KRUX_OK || done) return gs;
    dl->base = -1;
  }
  constexpr int W = kMaxN / 64;
  std::vector<int64_t> idx(m);
  std::vector<uint64_t> mask((size_t)m * W);
  KRUX_CUDA(ctx, cudaMemcpyAsync(idx.data(), ctx->miss_idx.p, m * 8, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(mask.data(), ctx->miss_mask.p, mask.size() * 8,
                                 cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  // the slots in SNP order (each SNP has at most one slot) and the complete rows,
  // by one placement pass instead of a sort
  std::vector<int32_t> slot_of((size_t)n, -1);
  for (int64_t i = 0; i < m; ++i) slot_of[(size_t)(idx[i] - b)] = (int32_t)i;
  std::vector<int64_t> order;
  order.reserve((size_t)m);
  complete.reserve((size_t)(n - m));
  for (int64_t j = 0; j < n; ++j) {
    if (slot_of[(size_t)j] >= 0) order.push_back(slot_of[(size_t)j]);
    else complete.push_back(b + j);
  }
  // buckets in order of their first SNP, found through an open-addressing table of
  // 64-bit mask hashes (a hash match is confirmed on the whole mask)
  auto mask_of = [&](int64_t oi) { return mask.data() + (size_t)oi * W; };
  auto hash_of = [&](const uint64_t *k) {
    uint64_t h = 0x9e3779b97f4a7c15ull;
    for (int w = 0; w < W; ++w) h = (h ^ k[w]) * 0x100000001b3ull;
    return h ^ (h >> 29);
  };
  size_t cap = 16;
  while (cap < 2 * (size_t)m) cap <<= 1;
  std::vector<int64_t> table(cap, -1);       // bucket index, -1 = empty
  std::vector<int64_t> first;                // each bucket's first slot (its mask)
  std::vector<uint64_t> hashes;              // and its hash
  for (int64_t oi : order) {
    const uint64_t *key = mask_of(oi);
    const uint64_t h = hash_of(key);
    size_t t = (size_t)h & (cap - 1);
    int64_t bi = -1;
    while (table[t] >= 0) {
      const int64_t c = table[t];
      if (hashes[(size_t)c] == h && std::memcmp(mask_of(first[(size_t)c]), key, W * 8) == 0) {
        bi = c;
        break;
      }
      t = (t + 1) & (cap - 1);
    }
    if (bi < 0) {
      bi = (int64_t)buckets.size();
      table[t] = bi;
      first.push_back(oi);
      hashes.push_back(h);
      Bucket bk;
      for (int k = 0; k < N; ++k)
        if ((key[k / 64] >> (k % 64)) & 1ull) bk.drop.push_back(k);
      buckets.push_back(std::move(bk));
    }
    buckets[(size_t)bi].snps.push_back(idx[oi]);
  }
  return KRUX_OK;
}

}  // namespace

// ------------------------------------------------------------------------------
// Scan groups and hit-list slots.
namespace {

// One output hit list.  Groups writing the same slot share its counter, so the
// list is one contiguous array whatever the number of groups.
struct OutSlot {
  krux_hit *hits = nullptr;
  double *H = nullptr, *P = nullptr;
  int64_t capacity = 0;
  HitAux *aux = nullptr;
  HitAux2 *aux2 = nullptr;  // markers with more than three groups (set by prepare_fused)
};

struct ScanGroupIn {
  const krux_rankset *rs = nullptr;  // geometry (T, N, Np, rows_pad)
  const __half *A = nullptr;         // n_agroups stacked rank matrices of rows_pad rows
  int n_agroups = 1;
  const float *tau = nullptr;
  const double *cfac = nullptr;
  const uint32_t *tile_nan = nullptr;
  const uint16_t *nan_cnt = nullptr;  // nullptr when no trait has NaN
  const uint16_t *nan_idx = nullptr;
  int64_t nan_ag_stride = 0;          // permuted groups: elements between agroups' NaN lists
  const int8_t *geno = nullptr;
  int64_t ldg = 0;
  const int64_t *snp_list = nullptr;  // device rows, or nullptr for [snp_begin, +n_snps)
  int64_t list_off = -1;              // offset into the call's list buffer (patched later)
  int64_t snp_begin = 0, n_snps = 0;
  int allow_missing = 0;
  int out_slot = 0;
  double *dense_H = nullptr, *dense_p = nullptr;
  int64_t dense_ld = 0, dense_snp0 = 0;
  double *minp_key = nullptr;
  unsigned long long *minp_bound = nullptr;  // the plain form's bounds beside the keys
  unsigned long long *minp_seed = nullptr;  // and its seed pass's records
  int bucket = -1;                    // index into the call's bucket rank sets
  // tensor map of A: groups whose rank matrices sit back to back in one buffer
  // (missing-pattern buckets of one rank set) share it, each at row a_row0
  const __half *a_map = nullptr;      // nullptr: a map of A's own rows
  int64_t a_map_rows = 0, a_row0 = 0;
};

struct BucketJob {
  const krux_rankset *base;
  std::vector<int32_t> drop;
};

// All state of one scan call that must outlive the launch.
struct CallPlan {
  std::vector<ScanGroupIn> groups;
  std::vector<OutSlot> slots;
  std::vector<int64_t> lists;         // host copy of all SNP lists
  std::vector<BucketJob> bucket_jobs;
  std::vector<krux_rankset> bucket_sets;  // host shells of the re-ranked sets
  struct PermJob {  // permutation batch: the stacked, permuted rank matrices
    bool on = false;
    const krux_rankset *rs = nullptr;
    const int32_t *perms = nullptr;
    int P = 0;
    __half *stack = nullptr;     // [1 + P][rows_pad][Np]
    double *minp = nullptr;      // caller's [P][T]
    uint16_t *lists = nullptr;   // [1 + P][T][N] NaN sample lists (rank sets with NaN)
    int32_t *inv = nullptr;      // [P][N] inverse permutations
    bool pre_done = false;       // the stacking was queued already (before a seed pass)
    bool seed = false;           // min-p seed pass: permuted agroups only, no hits, no FDR
  } perm;
  bool multi = false;  // markers with codes 0..4 (chunks of kChunkSnpsM SNPs)
  struct Param {  // parametric comparison: fused test bounds and the FP64 decision
    int model = -1;                 // -1 off, 0 ANOVA, 1 dosage regression
    double h1 = 0.0, h2 = 0.0;      // ANOVA bounds tau_1, tau_2 on sum_i S_i^2 / N_i
    double rl = 0.0;                // regression: 1 / ((K - 1) r_c^2)
    const float *expr = nullptr;    // the caller's values, for the FP64 recomputation
    int64_t ld = 0;
    const double *mean = nullptr;   // per-trait mean the recomputation centres on
    krux_hit *out = nullptr;        // the caller's lists
    double *out_stat = nullptr, *out_p = nullptr;
    int64_t out_capacity = 0;
  } param;
  struct Cis {  // cis scans: SNP and trait coordinates (host copies) and the window
    bool on = false;
    const int64_t *snp_pos = nullptr, *trait_pos = nullptr;  // device
    std::vector<int64_t> h_snp, h_trait;                      // host copies
    int64_t window = -1;
  } cis;
  int64_t dlist_used = 0;  // entries of ctx->dlist this call's device groupings use
  unsigned long long *fdr_hist = nullptr;  // permutation calls: [fdr_rows = 1 + P][fdr_bins] or null
  int fdr_rows = 0, fdr_bins = 0;
  double fdr_l0 = 0.0, fdr_w = 1.0;
};

// Device bytes of one bucket's re-ranked set apart from A (tie sums, K, tau, cfac);
// the A matrices of a call's buckets lie back to back before these.
size_t bucket_bytes(const krux_rankset *rs) {
  size_t off = 0;
  auto take = [&](size_t b) { off += (b + 255) / 256 * 256; };
  take((size_t)rs->T * 8);
  take((size_t)rs->T * 4);
  take((size_t)rs->rows_pad * 4);
  take((size_t)rs->rows_pad * 8);
  return off;
}

// Groups for one rank set against SNP rows [b, e) of geno: complete SNPs as one
// group, and one group per missing-sample pattern (section "Handling missing
// values").  A / n_agroups give the (possibly permutation-stacked) rank matrices.
krux_status plan_groups(krux_ctx *ctx, CallPlan &cp, const krux_rankset *rs, const int8_t *geno,
                        int64_t ldg, int64_t b, int64_t e, const __half *A, int n_agroups,
                        int slot, double *dense_H, double *dense_p, double *minp_key,
                        cudaStream_t s) {
  const int64_t n = e - b;
  if (n <= 0) return KRUX_OK;
  std::vector<Bucket> buckets;
  std::vector<int64_t> complete;
  bool bad = false;
  DevLists dl;
  if ((int64_t)(ctx->dlist.n / 8) >= cp.dlist_used + n) dl.base = cp.dlist_used;
  krux_status st = find_missing(ctx, geno, ldg, rs->N, b, n, s, buckets, complete, bad,
                                cp.multi ? kMaxCodeM : 2, &dl);
  if (st != KRUX_OK) return st;
  if (dl.base >= 0 && !buckets.empty()) cp.dlist_used += n;
  if (bad)
    return fail(ctx, KRUX_EINVAL, cp.multi ? "genotype code outside {-1, 0..4}"
                                           : "genotype code outside {-1,0,1,2}");
  if (cp.multi && rs->has_nan)
    return fail(ctx, KRUX_EUNSUPPORTED, "markers with more than three groups need complete expression");
  if (!buckets.empty() && n_agroups > 1)
    return fail(ctx, KRUX_EUNSUPPORTED, "permutation scan with missing genotypes");
  ScanGroupIn g0;
  g0.rs = rs;
  g0.A = A ? A : rs->dev.A;
  g0.n_agroups = n_agroups;
  g0.tau = rs->dev.tau;
  g0.cfac = rs->dev.cfac;
  g0.tile_nan = rs->dev.tile_nan;
  g0.nan_cnt = rs->has_nan ? rs->dev.nan_cnt : nullptr;
  g0.nan_idx = rs->dev.nan_idx;
  g0.geno = geno;
  g0.ldg = ldg;
  g0.out_slot = slot;
  g0.dense_H = dense_H;
  g0.dense_p = dense_p;
  g0.dense_ld = n;
  g0.dense_snp0 = b;
  g0.minp_key = minp_key;
  if (buckets.empty()) {
    g0.snp_begin = b;
    g0.n_snps = n;
    cp.groups.push_back(g0);
    return KRUX_OK;
  }
  if (dl.base >= 0 && dl.complete_count > 0) {  // device lists
    g0.snp_list = ctx->dlist.as<int64_t>() + dl.complete_off;
    g0.n_snps = dl.complete_count;
    cp.groups.push_back(g0);
  } else if (!complete.empty()) {
    g0.list_off = (int64_t)cp.lists.size();
    g0.n_snps = (int64_t)complete.size();
    cp.lists.insert(cp.lists.end(), complete.begin(), complete.end());
    cp.groups.push_back(g0);
  }
  for (auto &bk : buckets) {
    ScanGroupIn gb = g0;
    gb.minp_key = nullptr;
    if (bk.dev_off >= 0) {
      gb.list_off = -1;
      gb.snp_list = ctx->dlist.as<int64_t>() + bk.dev_off;
      gb.n_snps = bk.count;
      gb.allow_missing = 1;
      gb.bucket = (int)cp.bucket_jobs.size();
      cp.bucket_jobs.push_back(BucketJob{rs, bk.drop});
      cp.groups.push_back(gb);
      continue;
    }
    gb.list_off = (int64_t)cp.lists.size();
    gb.n_snps = (int64_t)bk.snps.size();
    gb.allow_missing = 1;
    gb.bucket = (int)cp.bucket_jobs.size();
    cp.lists.insert(cp.lists.end(), bk.snps.begin(), bk.snps.end());
    cp.bucket_jobs.push_back(BucketJob{rs, bk.drop});
    cp.groups.push_back(gb);
  }
  return KRUX_OK;
}

// Uploads SNP lists, re-ranks every bucket, and points the groups at the results.
krux_status materialise(krux_ctx *ctx, CallPlan &cp, cudaStream_t s) {
  if (!cp.lists.empty()) {
    KRUX_CUDA(ctx, ctx->list.ensure(cp.lists.size() * 8));
    KRUX_CUDA(ctx, ctx->list_host.ensure(cp.lists.size() * 8));
    std::memcpy(ctx->list_host.p, cp.lists.data(), cp.lists.size() * 8);
    KRUX_CUDA(ctx, cudaMemcpyAsync(ctx->list.p, ctx->list_host.p, cp.lists.size() * 8,
                                   cudaMemcpyHostToDevice, s));
  }
  for (auto &g : cp.groups)
    if (g.list_off >= 0) g.snp_list = ctx->list.as<int64_t>() + g.list_off;
  if (cp.bucket_jobs.empty()) return KRUX_OK;
  const size_t nb = cp.bucket_jobs.size();
  std::vector<size_t> aoff(nb), off(nb);
  size_t tot = 0;
  for (size_t i = 0; i < nb; ++i) {  // rows_pad * Np * 2 is a multiple of 256
    aoff[i] = tot;
    tot += (size_t)cp.bucket_jobs[i].base->rows_pad * cp.bucket_jobs[i].base->Np * 2;
  }
  for (size_t i = 0; i < nb; ++i) {
    off[i] = tot;
    tot += bucket_bytes(cp.bucket_jobs[i].base);
  }
  std::vector<int32_t> drops;
  std::vector<RerankJob> jobs(nb);
  for (size_t i = 0; i < nb; ++i) {
    jobs[i].drop_off = (int32_t)drops.size();
    jobs[i].n_drop = (int32_t)cp.bucket_jobs[i].drop.size();
    drops.insert(drops.end(), cp.bucket_jobs[i].drop.begin(), cp.bucket_jobs[i].drop.end());
  }
  if (drops.empty()) drops.push_back(0);
  const size_t jobs_off = tot;
  tot += (nb * sizeof(RerankJob) + 255) / 256 * 256;
  const size_t drop_off = tot;
  tot += drops.size() * 4;
  KRUX_CUDA(ctx, ctx->bucket_ranks.ensure(tot));
  char *base = ctx->bucket_ranks.as<char>();
  cp.bucket_sets.assign(nb, krux_rankset());
  for (size_t i = 0; i < nb; ++i) {
    const krux_rankset *rs = cp.bucket_jobs[i].base;
    krux_rankset &bs = cp.bucket_sets[i];
    bs.T = rs->T;
    bs.N = rs->N;
    bs.Np = rs->Np;
    bs.rows_pad = rs->rows_pad;
    bs.n_ttiles = rs->n_ttiles;
    bs.has_nan = rs->has_nan;
    bs.nan_traits_over = rs->nan_traits_over;
    char *p = base + off[i];
    size_t o2 = 0;
    auto take = [&](size_t bytes) {
      char *r = p + o2;
      o2 += (bytes + 255) / 256 * 256;
      return r;
    };
    bs.dev.A = reinterpret_cast<__half *>(base + aoff[i]);
    bs.dev.tie = (int64_t *)take((size_t)rs->T * 8);
    bs.dev.K = (int32_t *)take((size_t)rs->T * 4);
    bs.dev.tau = (float *)take((size_t)rs->rows_pad * 4);
    bs.dev.cfac = (double *)take((size_t)rs->rows_pad * 8);
    // dropping samples with a missing genotype leaves the NaN samples as they are
    bs.dev.nan_cnt = rs->dev.nan_cnt;
    bs.dev.nan_idx = rs->dev.nan_idx;
    bs.dev.tile_nan = rs->dev.tile_nan;
    RerankJob &j = jobs[i];
    j.base = rs->dev;
    j.A = bs.dev.A;
    j.tie = bs.dev.tie;
    j.K = bs.dev.K;
    j.tau = bs.dev.tau;
    j.cfac = bs.dev.cfac;
    j.T = rs->T;
    j.N = rs->N;
    j.Np = rs->Np;
    j.rows_pad = rs->rows_pad;
  }
  // pageable uploads: staged before the calls return, so the host vectors may go
  RerankJob *djobs = reinterpret_cast<RerankJob *>(base + jobs_off);
  int32_t *ddrop = reinterpret_cast<int32_t *>(base + drop_off);
  KRUX_CUDA(ctx, cudaMemcpyAsync(djobs, jobs.data(), nb * sizeof(RerankJob), cudaMemcpyHostToDevice, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(ddrop, drops.data(), drops.size() * 4, cudaMemcpyHostToDevice, s));
  KRUX_CUDA(ctx, launch_rerank_buckets(djobs, jobs.data(), ddrop, (int)nb, s));
  if (ctx->profiling) ctx->prof.launches += 1;
  // runs of buckets of the same rank set: one A map each
  std::vector<size_t> run(nb);
  for (size_t i = 0; i < nb; ++i)
    run[i] = (i > 0 && cp.bucket_jobs[i].base == cp.bucket_jobs[i - 1].base) ? run[i - 1] : i;
  std::vector<int64_t> run_rows(nb, 0);
  for (size_t i = 0; i < nb; ++i) run_rows[run[i]] += cp.bucket_jobs[i].base->rows_pad;
  for (auto &g : cp.groups) {
    if (g.bucket < 0) continue;
    const krux_rankset &bs = cp.bucket_sets[g.bucket];
    const size_t r = run[(size_t)g.bucket];
    g.a_map = reinterpret_cast<const __half *>(base + aoff[r]);
    g.a_map_rows = run_rows[r];
    g.a_row0 = (int64_t)((aoff[(size_t)g.bucket] - aoff[r]) / ((size_t)bs.Np * 2));
    g.A = bs.dev.A;
    g.tau = bs.dev.tau;
    g.cfac = bs.dev.cfac;
    g.tile_nan = bs.dev.tile_nan;
    g.nan_cnt = bs.has_nan ? bs.dev.nan_cnt : nullptr;
    g.nan_idx = bs.dev.nan_idx;
  }
  return KRUX_OK;
}

// cis scans: for every B tile, only the trait tiles whose traits can lie within
// the window of one of the tile's SNPs (SNP and trait coordinates are
// nondecreasing, so that is one contiguous range of trait tiles); B tiles with
// none are skipped.
std::vector<WorkItem> make_items_cis(const CallPlan &cp, const std::vector<GroupPlan> &gp) {
  std::vector<WorkItem> items;
  const std::vector<int64_t> &tp = cp.cis.h_trait;
  const int64_t W = cp.cis.window;
  for (size_t gi = 0; gi < gp.size(); ++gi) {
    const ScanGroupIn &g = cp.groups[gi];
    const GroupDesc &d = gp[gi].d;
    auto snp_at = [&](int64_t i) {
      return g.list_off >= 0 ? cp.lists[(size_t)(g.list_off + i)] : g.snp_begin + i;
    };
    for (int64_t b = 0; b < gp[gi].n_btiles; ++b) {
      const int64_t csn = cp.multi ? kChunkSnpsM : kChunkSnps;
      const int64_t first = b * d.nc * csn;
      const int64_t last = std::min<int64_t>((b + 1) * d.nc * csn, g.n_snps) - 1;
      if (first > last) continue;
      const int64_t lo = cp.cis.h_snp[(size_t)snp_at(first)] - W;
      const int64_t hi = cp.cis.h_snp[(size_t)snp_at(last)] + W;
      const int64_t t0 = std::lower_bound(tp.begin(), tp.end(), lo) - tp.begin();
      const int64_t t1 = std::upper_bound(tp.begin(), tp.end(), hi) - tp.begin();
      if (t0 >= t1) continue;
      WorkItem w;
      w.group = (int32_t)gi;
      w.btile = (int32_t)b;
      w.step_begin = (int32_t)(t0 / kTileM);
      w.step_end = (int32_t)((t1 - 1) / kTileM + 1);
      items.push_back(w);
    }
  }
  return items;
}

// One fused launch, split in three phases so that the middle one can be captured
// in a CUDA graph: prepare (host planning, buffer sizing, descriptor uploads; no
// work queued that a replay would need), enqueue (stream work only: packing, the
// scan, compaction, device-count-driven finalisation), finish (synchronise, read
// the counts and the status word).
struct FusedLaunch {
  ScanParams p{};
  int grid = 0;
  size_t smem = 0;
  bool staged = false;
  int n_seg = 0;
  int nslots = 0;
  double h1 = 0.0, h2 = 0.0;
  int signed_coef = 0;
  bool fast_nan = false;  // the plain form's NaN variant (coefficient sets in the codes)
  std::vector<int64_t> boff, moff, coff;
  int layout = 1;
  double hm[4] = {0.0, 0.0, 0.0, 0.0};  // markers with codes 0..4: h_d for d = 1..4
  // biallelic rank-sum groups: all packed by one launch (job table on the device)
  bool batched_pack = false;
  int n_pack_jobs = 0;
  int64_t pack_slots = 0, pack_halves = 0;
  const PackJob *packjobs = nullptr;        // this launch's tables (device)
  const double *const *cfacptr = nullptr;
};

// tables = 1 puts this launch's tables (group descriptors, work items, pack jobs,
// tie-factor pointers) in the context's second set, so that two prepared launches
// can be enqueued back to back without a host synchronisation between them.
// allow_fast_nan = false keeps a call with NaN expression in the general form (the
// plan is made again that way when the plain form's NaN variant does not fit).
krux_status prepare_fused(krux_ctx *ctx, CallPlan &cp, const krux_opts *o, FusedLaunch &fl,
                          cudaStream_t s, int tables = 0, bool allow_fast_nan = true) {
  DevBuf &t_groups = tables ? ctx->groups2 : ctx->groups;
  DevBuf &t_items = tables ? ctx->items2 : ctx->items;
  DevBuf &t_packjobs = tables ? ctx->packjobs2 : ctx->packjobs;
  DevBuf &t_cfacptr = tables ? ctx->cfacptr2 : ctx->cfacptr;
  fl.h1 = cp.param.model == 0 ? cp.param.h1 : h_df1(o->pthresh);
  fl.h2 = cp.param.model == 0 ? cp.param.h2 : h_df2(o->pthresh);
  const int ng = (int)cp.groups.size();
  fl.nslots = (int)cp.slots.size();
  fl.signed_coef = 0;
  for (auto &g : cp.groups) fl.signed_coef |= g.minp_key != nullptr ? 1 : 0;
  KRUX_CUDA(ctx, ctx->counters.ensure((size_t)fl.nslots * 16 + 64));
  KRUX_CUDA(ctx, ctx->status.ensure(64));
  if (ng == 0) return KRUX_OK;
  int lay = -1, tnc = ctx->tune_nc, tnA = ctx->tune_nA, tka = ctx->tune_ka;
  const int atom0 = layout_atom(ctx->tune_layout >= 0 ? ctx->tune_layout : 1);
  int kpad0 = atom0;
  for (auto &g : cp.groups) kpad0 = std::max(kpad0, round_up(g.rs->Np, atom0));
  if (ctx->tune_layout >= 0 || ctx->tune_nc > 0) {
    lay = ctx->tune_layout;
  } else {
    // a shape picked by krux_autotune for this width, if there is one
    auto it = ctx->tuned.find(round_up(kpad0, 16));
    if (it != ctx->tuned.end()) {
      lay = it->second[0];
      tnc = it->second[1];
      tnA = it->second[2];
      tka = it->second[3];
    }
  }
  const int layout = lay >= 0 ? lay : 1;
  fl.layout = layout;
  const int atom = layout_atom(layout);
  // a call that can take the plain form keeps room for its hit-event ring; with
  // NaN expression it takes the form's NaN variant (per-chunk coefficient sets in
  // place of the 2-bit codes) when at most one trait in 128 has more NaN samples
  // than the last set covers (each such trait sends all its pairs to the exact
  // test; beyond that share the general form is faster)
  bool fast_shape = layout == 1 && !cp.multi && cp.param.model < 0 && o->dense_H == nullptr &&
                    !cp.cis.on;
  bool any_nan = false, fast_nan = allow_fast_nan && fast_shape;
  for (auto &g : cp.groups) {
    fast_nan = fast_nan && g.minp_key == nullptr &&
               (g.nan_cnt == nullptr || 128 * g.rs->nan_traits_over <= g.rs->T);
    any_nan = any_nan || g.nan_cnt != nullptr;
  }
  fast_nan = fast_nan && any_nan;
  fast_shape = fast_shape && (!any_nan || fast_nan);
  fl.fast_nan = fast_nan;
  int kpad = atom, codes_k = 0;
  for (auto &g : cp.groups) {
    kpad = std::max(kpad, round_up(g.rs->Np, atom));
    if (g.nan_cnt) codes_k = std::max(codes_k, fast_nan ? kCoefNanRows : g.rs->Np);
  }
  LaunchShape sh;
  {
    const int s_nc = ctx->tune_nc, s_nA = ctx->tune_nA, s_ka = ctx->tune_ka;
    ctx->tune_nc = tnc;
    ctx->tune_nA = tnA;
    ctx->tune_ka = tka;
    const bool ok = pick_launch_shape(ctx, kpad, codes_k, sh, fast_shape ? kEvRegion : 0);
    ctx->tune_nc = s_nc;
    ctx->tune_nA = s_nA;
    ctx->tune_ka = s_ka;
    if (!ok)
      return fail(ctx, tnc > 0 ? KRUX_EINVAL : KRUX_EUNSUPPORTED,
                  "no pipeline shape fits shared memory (Np=%d, tuning nc=%d nA=%d ka=%d)", kpad,
                  tnc, tnA, tka);
  }
  fl.boff.assign(ng, 0);
  fl.moff.assign(ng, 0);
  fl.coff.assign(ng, 0);
  int64_t btot = 0, mtot = 0, ctot = 0;
  for (int i = 0; i < ng; ++i) {
    const int64_t csn = cp.multi ? kChunkSnpsM : kChunkSnps;
    const int64_t nch = (cp.groups[i].n_snps + csn - 1) / csn;
    fl.boff[i] = btot;
    fl.moff[i] = mtot;
    fl.coff[i] = ctot;
    btot += (nch * kChunkRows * cp.groups[i].rs->Np * 2 + 255) / 256 * 256;
    mtot += nch;
    if (cp.groups[i].nan_cnt) ctot += nch * (fast_nan ? kCoefNanRows : cp.groups[i].rs->Np) * 2;
  }
  KRUX_CUDA(ctx, ctx->B.ensure(std::max<int64_t>(btot, 256)));
  if (cp.multi) {  // second side records, at the same offsets as the first
    const HitAux *base = ctx->aux.as<HitAux>();
    int64_t total = 1;
    for (auto &os : cp.slots)
      total = std::max<int64_t>(total, (int64_t)(os.aux - base) + std::max<int64_t>(os.capacity, 1));
    KRUX_CUDA(ctx, ctx->aux2.ensure((size_t)total * sizeof(HitAux2)));
    for (auto &os : cp.slots) os.aux2 = ctx->aux2.as<HitAux2>() + (os.aux - base);
    for (int d = 1; d <= 4; ++d) fl.hm[d - 1] = h_dfk(o->pthresh, d);
  }
  KRUX_CUDA(ctx, ctx->meta.ensure(std::max<int64_t>(mtot, 1) * sizeof(ChunkMeta)));
  KRUX_CUDA(ctx, ctx->codes.ensure(std::max<int64_t>(ctot, 1) * 8));
  std::vector<GroupDesc> descs(ng);
  std::vector<GroupPlan> plans(ng);
  int nc_max = 1;
  // encoded maps by (base, width, rows): groups in one buffer share a map
  std::map<std::tuple<const void *, int, int64_t>, CUtensorMap> maps;
  auto map_of = [&](CUtensorMap *out, const void *base, int Np, int64_t rows) -> krux_status {
    const auto key = std::make_tuple(base, Np, rows);
    auto it = maps.find(key);
    if (it == maps.end()) {
      CUtensorMap m;
      const krux_status st = encode_map(ctx, &m, base, Np, rows, layout);
      if (st != KRUX_OK) return st;
      it = maps.emplace(key, m).first;
    }
    *out = it->second;
    return KRUX_OK;
  };
  for (int i = 0; i < ng; ++i) {
    ScanGroupIn &g = cp.groups[i];
    const krux_rankset *rs = g.rs;
    const OutSlot &os = cp.slots[g.out_slot];
    __half *B = reinterpret_cast<__half *>(ctx->B.as<char>() + fl.boff[i]);
    GroupDesc &d = plans[i].d;
    std::memset(&d, 0, sizeof d);
    const int64_t csn = cp.multi ? kChunkSnpsM : kChunkSnps;
    const int64_t nch = (g.n_snps + csn - 1) / csn;
    krux_status st;
    if (g.a_map) {
      st = map_of(&d.tmA, g.a_map, rs->Np, g.a_map_rows);
      d.a_row0 = (int32_t)g.a_row0;
    } else {
      st = map_of(&d.tmA, g.A, rs->Np, (int64_t)rs->rows_pad * g.n_agroups);
    }
    if (st != KRUX_OK) return st;
    const int64_t pitch = (int64_t)rs->Np * 2;  // bytes per B row
    if (fl.boff[i] % pitch == 0) {  // the whole B buffer as rows of this width
      st = map_of(&d.tmB, ctx->B.p, rs->Np, std::max<int64_t>(btot / pitch, 1));
      d.b_row0 = (int32_t)(fl.boff[i] / pitch);
    } else {
      st = map_of(&d.tmB, B, rs->Np, std::max<int64_t>(nch, 1) * kChunkRows);
    }
    if (st != KRUX_OK) return st;
    d.meta = ctx->meta.as<ChunkMeta>() + fl.moff[i];
    d.codes = g.nan_cnt ? ctx->codes.as<uint64_t>() + fl.coff[i] : nullptr;
    d.codes_k = g.nan_cnt ? (fast_nan ? kCoefNanRows : rs->Np) : 0;
    d.geno = g.geno;
    d.ldg = g.ldg;
    d.tau = g.tau;
    d.cfac = g.cfac;
    d.nan_cnt = g.nan_cnt;
    d.nan_idx = g.nan_idx;
    d.nan_ag_stride = g.nan_ag_stride;
    d.tile_nan = g.tile_nan;
    d.hits = os.hits;
    d.aux = os.aux;
    d.aux2 = os.aux2;
    d.counter = ctx->counters.as<unsigned long long>() + g.out_slot;
    d.capacity = os.capacity;
    d.dense_H = g.dense_H;
    d.dense_p = g.dense_p;
    d.dense_ld = g.dense_ld;
    d.dense_snp0 = g.dense_snp0;
    d.minp_key = g.minp_key;
    d.minp_bound = g.minp_bound;
    d.minp_seed = g.minp_seed;
    d.T = rs->T;
    d.N = rs->N;
    d.Np = rs->Np;
    d.n_ttiles = rs->n_ttiles;
    d.rows_per_agroup = rs->rows_pad;
    d.n_agroups = g.n_agroups;
    d.nchunks = (int32_t)nch;
    d.n_atoms = (rs->Np + atom - 1) / atom;
    d.group_id = i;
    group_shape(sh, round_up(rs->Np, atom), atom, d);
    nc_max = std::max(nc_max, d.nc);
    plans[i].n_btiles = (nch + d.nc - 1) / d.nc;
    plans[i].steps = (int64_t)g.n_agroups * rs->n_ttiles;
    if (cp.perm.seed) plans[i].step_lo = rs->n_ttiles;
    descs[i] = d;
  }
  std::vector<WorkItem> items =
      cp.cis.on ? make_items_cis(cp, plans) : make_items(plans, nc_max, ctx->sm_count);
  KRUX_CUDA(ctx, t_groups.ensure(sizeof(GroupDesc) * ng));
  KRUX_CUDA(ctx, t_items.ensure(sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
  // pageable uploads: staged before the calls return, so the host vectors may go
  KRUX_CUDA(ctx, cudaMemcpyAsync(t_groups.p, descs.data(), sizeof(GroupDesc) * ng,
                                 cudaMemcpyHostToDevice, s));
  if (!items.empty())
    KRUX_CUDA(ctx, cudaMemcpyAsync(t_items.p, items.data(), sizeof(WorkItem) * items.size(),
                                   cudaMemcpyHostToDevice, s));
  fl.batched_pack = !cp.multi && cp.param.model != 1;
  if (fl.batched_pack) {
    std::vector<PackJob> jobs(ng);
    int64_t slots = 0, halves = 0;
    for (int i = 0; i < ng; ++i) {
      const ScanGroupIn &g = cp.groups[i];
      PackJob &j = jobs[i];
      std::memset(&j, 0, sizeof j);
      const int64_t nch = (g.n_snps + kChunkSnps - 1) / kChunkSnps;
      j.geno = g.geno;
      j.ldg = g.ldg;
      j.snp_list = g.snp_list;
      j.snp_begin = g.snp_begin;
      j.n_snps = g.n_snps;
      j.slot0 = slots;
      j.half0 = halves;
      j.B = reinterpret_cast<__half *>(ctx->B.as<char>() + fl.boff[i]);
      j.meta = ctx->meta.as<ChunkMeta>() + fl.moff[i];
      j.codes = g.nan_cnt ? ctx->codes.as<uint64_t>() + fl.coff[i] : nullptr;
      j.N = g.rs->N;
      j.Np = g.rs->Np;
      j.allow_missing = g.allow_missing;
      j.coef_nan = j.codes != nullptr && fast_nan ? 1 : 0;
      slots += nch * kChunkSnps;
      if (j.codes && !j.coef_nan) halves += nch * 2;
    }
    fl.n_pack_jobs = ng;
    fl.pack_slots = slots;
    fl.pack_halves = halves;
    KRUX_CUDA(ctx, t_packjobs.ensure(sizeof(PackJob) * ng));
    KRUX_CUDA(ctx, cudaMemcpyAsync(t_packjobs.p, jobs.data(), sizeof(PackJob) * ng,
                                   cudaMemcpyHostToDevice, s));
    fl.packjobs = t_packjobs.as<PackJob>();
  }
  std::vector<const double *> cf(ng);
  for (int i = 0; i < ng; ++i) cf[i] = cp.groups[i].cfac;
  KRUX_CUDA(ctx, t_cfacptr.ensure(sizeof(double *) * ng));
  KRUX_CUDA(ctx, cudaMemcpyAsync(t_cfacptr.p, cf.data(), sizeof(double *) * ng,
                                 cudaMemcpyHostToDevice, s));
  fl.cfacptr = t_cfacptr.as<const double *>();
  KRUX_CUDA(ctx, finalize_prepare());
  ScanParams &p = fl.p;
  p = ScanParams{};
  p.groups = t_groups.as<GroupDesc>();
  p.items = t_items.as<WorkItem>();
  p.n_items = (int32_t)items.size();
  p.nc = nc_max;
  p.nA = sh.nA;
  p.kpad = std::max(codes_k, 16);
  p.ka = sh.ka;
  p.a_tile_bytes = 256 * sh.ka;
  p.b_region = sh.b_region;
  p.layout = layout;
  p.margin = (float)(o->recheck_margin > 0 ? o->recheck_margin : 1e-4);
  if (cp.param.model >= 0) {
    // FP16 standardised values: a wide band, every pair in it decided in FP64
    p.margin = 0.03f;
    p.provisional = 1;
  }
  p.dense = o->dense_H != nullptr ? 1 : 0;
  p.pthresh = o->pthresh;
  p.h1 = (float)fl.h1;
  p.h2 = (float)fl.h2;
  p.status = ctx->status.as<unsigned int>();
  p.timeout_cycles = ctx->wait_limit;
  p.signed_coef = fl.signed_coef;
  p.fdr_hist = cp.fdr_hist;
  p.fdr_bins = cp.fdr_bins;
  p.fdr_l0 = cp.fdr_l0;
  p.fdr_w = cp.fdr_w;
  p.multi = cp.multi ? 1 : 0;
  for (auto &g : cp.groups) p.perm |= g.minp_key != nullptr ? 1 : 0;
  p.seed_bound = cp.perm.seed ? 1 : 0;
  for (auto &g : cp.groups) p.has_nan |= g.nan_cnt != nullptr ? 1 : 0;
  if (cp.cis.on) {
    p.cis_snp_pos = cp.cis.snp_pos;
    p.cis_trait_pos = cp.cis.trait_pos;
    p.cis_window = cp.cis.window;
  }
  // the plain scan form: 32-byte swizzle, every group's chunks paired and its K
  // in one rank stage, complete data, no dense output, cis window, provisional
  // hits, permutations or markers with more than three groups
  {
    bool fast = layout == 1 && !p.multi && (!p.has_nan || fast_nan) && !p.dense && !p.provisional &&
                (!p.signed_coef || p.perm) && p.cis_window < 0;
    for (const GroupDesc &d : descs) fast = fast && d.pair == 1 && d.nkb == 1;
    p.fast = fast ? 1 : 0;
  }
  fl.grid = (int)std::min<size_t>(items.size(), (size_t)ctx->sm_count);
  // Single hit list: every epilogue warp stages its hits in a segment of its own
  // (no atomic per hit event) and the segments are appended after the launch.
  fl.staged = fl.nslots == 1 && cp.slots[0].capacity > 0 && fl.grid > 0;
  fl.n_seg = fl.grid * kEpiWarps;
  if (fl.staged) {
    const int64_t cap = cp.slots[0].capacity;
    const int seg_cap = (int)std::max<int64_t>(64, std::min<int64_t>(4096, 2 * cap / fl.n_seg + 64));
    const size_t rec = sizeof(krux_hit) + sizeof(HitAux);
    const size_t a2off = ((size_t)fl.n_seg * seg_cap * rec + (size_t)fl.n_seg * 4 + 255) / 256 * 256;
    const size_t a2 = cp.multi ? (size_t)fl.n_seg * seg_cap * sizeof(HitAux2) : 0;
    KRUX_CUDA(ctx, ctx->seg.ensure(a2off + a2 + 256));
    char *sb = ctx->seg.as<char>();
    p.seg_cap = seg_cap;
    p.seg_hits = reinterpret_cast<krux_hit *>(sb);
    p.seg_aux = reinterpret_cast<HitAux *>(sb + (size_t)fl.n_seg * seg_cap * sizeof(krux_hit));
    p.seg_cnt = reinterpret_cast<unsigned int *>(sb + (size_t)fl.n_seg * seg_cap * rec);
    if (cp.multi) p.seg_aux2 = reinterpret_cast<HitAux2 *>(sb + a2off);
  }
  fl.smem = scan_smem_bytes2(nc_max, sh.nA, (size_t)p.a_tile_bytes, (size_t)p.b_region, p.kpad);
  if (p.fast) {  // the plain scan form also holds its ring of hit-event buffers
    if (fl.smem + kEvRegion <= kSmemLimit) fl.smem += kEvRegion;
    else p.fast = 0;
  }
  if (fast_nan && !p.fast)  // the coefficient sets need the plain form: plan again
    return prepare_fused(ctx, cp, o, fl, s, tables, false);
  p.fast_nan = fast_nan ? 1 : 0;
  if (p.fast && p.perm && !cp.perm.seed && fl.grid > 0) {
    // each event warp's list for the deferred FP64 pass: about three times the
    // pairs a 200k-SNP batch passes on, at least 8192 and at most 65536 entries
    const int64_t per = (int64_t)48 * cp.perm.P * cp.perm.rs->rows_pad / (2 * fl.grid);
    const int cap = (int)std::min<int64_t>(65536, std::max<int64_t>(8192, per));
    const size_t lists = (size_t)2 * fl.grid * cap * sizeof(MinpPair);
    KRUX_CUDA(ctx, ctx->mcand.ensure(lists + (size_t)2 * fl.grid * 4 + 256));
    p.mc_list = ctx->mcand.as<MinpPair>();
    p.mc_cnt = reinterpret_cast<unsigned int *>(ctx->mcand.as<char>() + lists);
    p.mc_cap = cap;
  }
  const std::string why = validate_plan(p, descs, fl.smem);
  if (!why.empty()) return fail(ctx, KRUX_EUNSUPPORTED, "%s", why.c_str());
  if (fl.grid > 0) KRUX_CUDA(ctx, scan_set_smem(fl.smem));
  return KRUX_OK;
}

krux_status enqueue_fused(krux_ctx *ctx, CallPlan &cp, const FusedLaunch &fl, cudaStream_t s) {
  const int ng = (int)cp.groups.size();
  const int nslots = fl.nslots;
  KRUX_CUDA(ctx, cudaMemsetAsync(ctx->counters.p, 0, (size_t)nslots * 16 + 8, s));
  if (!cp.perm.pre_done)  // else the seed pass before this launch cleared it
    KRUX_CUDA(ctx, cudaMemsetAsync(ctx->status.p, 0, 64, s));
  if (cp.fdr_hist)
    KRUX_CUDA(ctx, cudaMemsetAsync(cp.fdr_hist, 0, (size_t)cp.fdr_rows * cp.fdr_bins * 8, s));
  if (ng == 0) {  // nothing to scan: a permutation batch still reports min p = 1
    if (cp.perm.on) {
      KRUX_CUDA(ctx, cudaMemsetAsync(ctx->minpkey.p, 0,
                                     (size_t)cp.perm.P * cp.perm.rs->rows_pad * 8, s));
      KRUX_CUDA(ctx, launch_minp_from_key(ctx->minpkey.as<double>(), cp.perm.minp, cp.perm.P,
                                          cp.perm.rs->T, cp.perm.rs->rows_pad, s));
    }
    return KRUX_OK;
  }
  unsigned int *status = ctx->status.as<unsigned int>();
  if (cp.perm.on && !cp.perm.pre_done) {
    const CallPlan::PermJob &pj = cp.perm;
    const krux_rankset *rs = pj.rs;
    const size_t one = (size_t)rs->rows_pad * rs->Np;
    KRUX_CUDA(ctx, cudaMemcpyAsync(pj.stack, rs->dev.A, one * 2, cudaMemcpyDeviceToDevice, s));
    KRUX_CUDA(ctx, launch_permute_rows(rs->dev.A, pj.stack + one, rs->rows_pad, rs->Np, rs->N,
                                       pj.perms, pj.P, status, s));
    KRUX_CUDA(ctx, cudaMemsetAsync(ctx->minpkey.p, 0, (size_t)pj.P * rs->rows_pad * 40, s));
    if (pj.lists) {
      // NaN samples of permutation q sit at inv_q(original position)
      const size_t lst = (size_t)rs->T * rs->N;
      // zero first: entries a bad replayed row never writes stay valid sample indices
      KRUX_CUDA(ctx, cudaMemsetAsync(pj.inv, 0, (size_t)pj.P * rs->N * 4, s));
      KRUX_CUDA(ctx, launch_invert_perms(pj.perms, pj.P, rs->N, pj.inv, s));
      KRUX_CUDA(ctx, cudaMemcpyAsync(pj.lists, rs->dev.nan_idx, lst * 2, cudaMemcpyDeviceToDevice, s));
      KRUX_CUDA(ctx, launch_permute_nan_idx(rs->dev.nan_cnt, rs->dev.nan_idx, rs->T, rs->N, pj.inv,
                                            pj.P, pj.lists + lst, s));
    }
  }
  ev_record(ctx, 2, s);
  if (fl.batched_pack)
    KRUX_CUDA(ctx, launch_pack_batch(fl.packjobs, fl.n_pack_jobs, fl.pack_slots,
                                     fl.pack_halves, fl.h1, fl.h2, fl.signed_coef, status, s));
  for (int i = 0; i < ng && !fl.batched_pack; ++i) {
    const ScanGroupIn &g = cp.groups[i];
    const krux_rankset *rs = g.rs;
    __half *B = reinterpret_cast<__half *>(ctx->B.as<char>() + fl.boff[i]);
    ChunkMeta *meta = ctx->meta.as<ChunkMeta>() + fl.moff[i];
    uint64_t *codes = g.nan_cnt ? ctx->codes.as<uint64_t>() + fl.coff[i] : nullptr;
    if (cp.param.model == 1)
      KRUX_CUDA(ctx, launch_pack_linear(g.geno, g.ldg, rs->N, rs->Np, g.snp_begin, g.n_snps,
                                        cp.param.rl, B, meta, status, s));
    else if (cp.multi)
      KRUX_CUDA(ctx, launch_pack_multi(g.geno, g.ldg, rs->N, rs->Np, g.snp_list, g.snp_begin,
                                       g.n_snps, fl.hm, g.allow_missing, B,
                                       reinterpret_cast<ChunkMetaM *>(meta), status, s));
    else
      KRUX_CUDA(ctx, launch_pack2(g.geno, g.ldg, rs->N, rs->Np, g.snp_list, g.snp_begin, g.n_snps,
                                  0, fl.h1, fl.h2, g.allow_missing, fl.signed_coef, B, meta, codes,
                                  status, s));
  }
  ev_record(ctx, 3, s);
  if (fl.p.mc_cnt)
    KRUX_CUDA(ctx, cudaMemsetAsync(fl.p.mc_cnt, 0, (size_t)2 * fl.grid * 4, s));
  ev_record(ctx, 7, s);  // the scan kernel alone: events 7 .. 4
  if (fl.grid > 0) KRUX_CUDA(ctx, launch_scan_only(fl.p, fl.grid, fl.smem, s));
  ev_record(ctx, 4, s);
  unsigned long long *totals = ctx->counters.as<unsigned long long>() + nslots;
  if (fl.staged) {
    KRUX_CUDA(ctx, launch_seg_compact(fl.p.seg_hits, fl.p.seg_aux, fl.p.seg_aux2, fl.p.seg_cnt,
                                      fl.n_seg, fl.p.seg_cap,
                                      ctx->counters.as<unsigned long long>(), cp.slots[0].hits,
                                      cp.slots[0].aux, cp.slots[0].aux2, cp.slots[0].capacity,
                                      totals, s));
  } else {
    KRUX_CUDA(ctx, cudaMemcpyAsync(totals, ctx->counters.p, (size_t)nslots * 8,
                                   cudaMemcpyDeviceToDevice, s));
  }
  // FP64 H and p of the stored hits: each slot's count is read on the device
  ev_record(ctx, 5, s);
  if (cp.param.model >= 0) {  // FP64 decision of the provisional hits, then the filter
    const OutSlot &os = cp.slots[0];
    const ScanGroupIn &g = cp.groups[0];
    KRUX_CUDA(ctx, launch_finalize_param(os.hits, totals, os.capacity, cp.param.expr, cp.param.ld,
                                         g.geno, g.ldg, g.rs->N, cp.param.mean, cp.param.model,
                                         os.H, os.P, ctx->sm_count, s));
    KRUX_CUDA(ctx, launch_filter_param(os.hits, totals, os.capacity, os.H, os.P, fl.p.pthresh,
                                       cp.param.out, cp.param.out_stat, cp.param.out_p,
                                       cp.param.out_capacity,
                                       ctx->counters.as<unsigned long long>() + 2 * nslots,
                                       ctx->sm_count, s));
  }
  for (int k = 0; k < nslots && cp.param.model < 0; ++k) {
    const OutSlot &os = cp.slots[k];
    if (os.capacity <= 0) continue;
    KRUX_CUDA(ctx, launch_finalize_dev(os.hits, os.aux, os.aux2, totals + k, os.capacity,
                                       fl.cfacptr, os.H, os.P,
                                       ctx->sm_count, s, cp.fdr_hist, cp.fdr_bins, cp.fdr_l0,
                                       cp.fdr_w, fl.p.pthresh));
  }
  ev_record(ctx, 6, s);
  if (fl.p.mc_list)  // the pairs the event warps passed on, decided in FP64
    KRUX_CUDA(ctx, launch_minp_cands(fl.p.mc_list, fl.p.mc_cnt, 2 * fl.grid, fl.p.mc_cap,
                                     cp.perm.rs->dev.cfac, cp.perm.rs->rows_pad, fl.p.pthresh,
                                     ctx->minpkey.as<double>(), cp.fdr_hist, cp.fdr_bins, cp.fdr_l0,
                                     cp.fdr_w, s));
  if (cp.perm.on && !cp.perm.seed)
    KRUX_CUDA(ctx, launch_minp_from_key(ctx->minpkey.as<double>(), cp.perm.minp, cp.perm.P,
                                        cp.perm.rs->T, cp.perm.rs->rows_pad, s));
  if (cp.perm.on && cp.perm.seed && fl.p.fast) {  // the plain form's seed records, decided
    const ScanGroupIn &g = cp.groups[0];
    const krux_rankset *rs = cp.perm.rs;
    KRUX_CUDA(ctx, launch_seed_decide(g.minp_seed, cp.perm.stack, rs->rows_pad, rs->Np, rs->N, rs->T,
                                      cp.perm.P, g.geno, g.ldg, g.snp_begin, g.n_snps,
                                      ctx->meta.as<ChunkMeta>() + fl.moff[0], rs->dev.cfac,
                                      g.minp_key, g.minp_bound, s));
  }
  return KRUX_OK;
}

int fused_launches(const CallPlan &cp, const FusedLaunch &fl) {
  int n = (fl.grid > 0 ? 1 : 0) + (fl.staged ? 1 : 0);
  if (fl.batched_pack)
    n += (fl.pack_slots > 0 ? 1 : 0) + (fl.pack_halves > 0 ? 1 : 0);
  else
    for (auto &g : cp.groups) n += g.nan_cnt ? 2 : 1;
  for (auto &os : cp.slots) n += (os.capacity > 0 && cp.param.model < 0) ? 1 : 0;
  if (cp.param.model >= 0) n += 2;
  if (cp.perm.on) {
    // the permuted stack (and NaN lists) unless a seed pass built them; then the
    // minimum-p read-out, or after a plain-form seed pass its exact decisions
    if (!cp.perm.pre_done) n += 1 + (cp.perm.lists ? 2 : 0);
    if (!cp.perm.seed || fl.p.fast) n += 1;
    if (fl.p.mc_list) n += 1;
  }
  return n;
}

// Reads the status word back; KRUX_OK, or the device-side error.
krux_status device_status(krux_ctx *ctx, const unsigned int *hst) {
  if (hst[0] & kDevBadCode) return fail(ctx, KRUX_EINVAL, "genotype code outside {-1,0,1,2}");
  if (hst[0] & kDevBadPerm) return fail(ctx, KRUX_EINVAL, "a permutation entry is outside 0..N-1");
  if (hst[0] & kDevTimeout)
    return fail(ctx, KRUX_ETIMEOUT, "device wait timed out (site %u)", hst[1]);
  return KRUX_OK;
}

krux_status finish_fused(krux_ctx *ctx, CallPlan &cp, const FusedLaunch &fl, cudaStream_t s,
                         std::vector<unsigned long long> &counts) {
  const int nslots = fl.nslots;
  counts.assign(nslots, 0);
  unsigned int hst[2] = {0, 0};
  if (!cp.groups.empty()) {
    KRUX_CUDA(ctx, cudaMemcpyAsync(counts.data(), ctx->counters.as<unsigned long long>() + nslots,
                                   (size_t)nslots * 8, cudaMemcpyDeviceToHost, s));
    KRUX_CUDA(ctx, cudaMemcpyAsync(hst, ctx->status.p, 8, cudaMemcpyDeviceToHost, s));
  }
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  if (ctx->profiling && !cp.groups.empty()) {
    ctx->prof.ms_pack = ev_ms(ctx, 2, 3);
    ctx->prof.ms_scan = ev_ms(ctx, 7, 4);
    ctx->prof.ms_finalize = ev_ms(ctx, 5, 6);
    ctx->prof.scan_grid = fl.grid;
    ctx->prof.scan_form = scan_form_of(fl.p);
    ctx->prof.launches += fused_launches(cp, fl);
  }
  return device_status(ctx, hst);
}

// Packs every group, launches the fused kernel once over all groups, finalises
// every slot's hits in FP64 and reads the per-slot hit counts back.
krux_status run_fused(krux_ctx *ctx, CallPlan &cp, const krux_opts *o, cudaStream_t s,
                      std::vector<unsigned long long> &counts) {
  FusedLaunch fl;
  krux_status st = prepare_fused(ctx, cp, o, fl, s);
  if (st != KRUX_OK) return st;
  st = enqueue_fused(ctx, cp, fl, s);
  if (st != KRUX_OK) return st;
  return finish_fused(ctx, cp, fl, s, counts);
}

// Seed pass of a permutation batch (section "P-value calculation and empirical
// FDR correction": the minimum p of each permuted trait over all SNPs): the
// permuted groups against the first kSeedSnps SNPs, so that the main launch
// starts from running minima over thousands of SNPs instead of none (without it
// the first wave of CTAs refines nearly every chunk in FP64).  False when the
// call is too small to gain from one.
bool make_seed_plan(const CallPlan &cp, CallPlan &seed, bool plain_form) {
  constexpr int64_t kSeedSnps = 16384;
  if (cp.groups.size() != 1) return false;
  const int64_t n = cp.groups[0].n_snps;
  // the plain form decides every pair past its bounds exactly, so its seed covers a
  // third of the SNPs (whole chunks; a quarter took 4 % longer over 200,000 SNPs at
  // P = 16, a sixth 7 %): few later pairs per class then beat the seed's best.  It
  // needs one at any size: from zero bounds nearly every pair of its first chunks
  // would go to the event warps (a 20,000-SNP batch took 83 ms without one)
  if (plain_form ? n < 16 * kChunkSnps : n <= 4 * kSeedSnps) return false;
  seed = cp;
  seed.groups[0].n_snps =
      plain_form ? std::max<int64_t>(4 * kChunkSnps, n / 3 / kChunkSnps * kChunkSnps) : kSeedSnps;
  seed.slots[0].capacity = 0;
  seed.fdr_hist = nullptr;
  seed.perm.seed = true;
  return true;
}

krux_status check_scan_args(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno, int64_t S,
                            int64_t ldg, const krux_opts *opts, krux_hit *hits, double *hit_H,
                            double *hit_p, int64_t *n_hits) {
  if (!ctx) return KRUX_EINVAL;
  if (!rs || !n_hits) return fail(ctx, KRUX_EINVAL, "NULL rank set or n_hits");
  krux_status st = check_opts(ctx, opts);
  if (st != KRUX_OK) return st;
  if (S < 0 || (S > 0 && ldg < rs->N)) return fail(ctx, KRUX_EINVAL, "need S >= 0 and ldg >= N");
  if (S > 0 && !geno) return fail(ctx, KRUX_EINVAL, "geno is NULL");
  if (S >= (int64_t)1 << 31) return fail(ctx, KRUX_EINVAL, "S must be < 2^31");
  if (opts->hit_capacity > 0 && (!hits || !hit_H || !hit_p))
    return fail(ctx, KRUX_EINVAL, "hit outputs are NULL");
  if (((uintptr_t)hits & 15u) != 0) return fail(ctx, KRUX_EINVAL, "hits must be 16-byte aligned");
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  if (b < 0 || e > S || b > e)
    return fail(ctx, KRUX_EINVAL, "bad SNP slice [%lld, %lld)", (long long)b, (long long)e);
  return KRUX_OK;
}

}  // namespace

extern "C" krux_status krux_scan(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                                 int64_t S, int64_t ldg, const krux_opts *opts, krux_hit *hits,
                                 double *hit_H, double *hit_p, int64_t *n_hits, void *stream) {
  krux_status st = check_scan_args(ctx, rs, geno, S, ldg, opts, hits, hit_H, hit_p, n_hits);
  if (st != KRUX_OK) return st;
  *n_hits = 0;
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    ctx->prof.pairs = (int64_t)rs->T * (e - b);
  }
  KRUX_CUDA(ctx, ctx->aux.ensure((size_t)std::max<int64_t>(opts->hit_capacity, 1) * sizeof(HitAux)));
  KRUX_CUDA(ctx, ctx->dlist.ensure((size_t)std::max<int64_t>(e - b, 1) * 8));
  CallPlan cp;
  cp.multi = (opts->flags & KRUX_FLAG_MULTIALLELIC) != 0;
  cp.slots.push_back(OutSlot{hits, hit_H, hit_p, opts->hit_capacity, ctx->aux.as<HitAux>()});
  st = plan_groups(ctx, cp, rs, geno, ldg, b, e, nullptr, 1, 0, opts->dense_H, opts->dense_p,
                   nullptr, s);
  if (st != KRUX_OK) return st;
  st = materialise(ctx, cp, s);
  if (st != KRUX_OK) return st;
  std::vector<unsigned long long> counts;
  st = run_fused(ctx, cp, opts, s, counts);
  if (st != KRUX_OK) return st;
  *n_hits = (int64_t)counts[0];
  if (*n_hits > opts->hit_capacity)
    return fail(ctx, KRUX_EOVERFLOW, "%lld hits exceed capacity %lld", (long long)*n_hits,
                (long long)opts->hit_capacity);
  return KRUX_OK;
}

// The device address of page-locked host memory mapped into the device's address
// space (cudaHostAlloc; cudaHostRegister with the mapped flag), else null.
static void *mapped_device_ptr(const void *host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();  // (an unknown pointer is not an error here)
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Host-memory wrapper of krux_rank + krux_scan: one copy per input into the
// context's device buffer (packed to leading dimension N), the scan into a
// device hit list the context keeps, and one copy per output array back.
extern "C" krux_status krux_scan_host(krux_ctx *ctx, const float *expr, int T, int N, int64_t lde,
                                      const int8_t *geno, int64_t S, int64_t ldg,
                                      const krux_opts *opts, krux_hit *hits, double *hit_H,
                                      double *hit_p, int64_t *n_hits, void *stream) {
  if (!ctx) return KRUX_EINVAL;
  if (!n_hits || !expr) return fail(ctx, KRUX_EINVAL, "NULL n_hits or expr");
  *n_hits = 0;
  krux_status st = check_opts(ctx, opts);
  if (st != KRUX_OK) return st;
  if (opts->dense_H || opts->dense_p)
    return fail(ctx, KRUX_EINVAL, "krux_scan_host: dense output is device-only (use krux_scan)");
  if (T < 1 || N < 1 || N > kMaxN || lde < N)
    return fail(ctx, KRUX_EINVAL, "krux_scan_host: need T >= 1, 1 <= N <= %d, lde >= N", kMaxN);
  if (S < 0 || (S > 0 && (ldg < N || !geno)))
    return fail(ctx, KRUX_EINVAL, "krux_scan_host: need S >= 0 and, for S > 0, geno and ldg >= N");
  if (opts->hit_capacity > 0 && (!hits || !hit_H || !hit_p))
    return fail(ctx, KRUX_EINVAL, "hit outputs are NULL");
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t ebytes = (size_t)T * N * 4, gbytes = (size_t)S * N;
  const size_t goff = (ebytes + 255) / 256 * 256;
  KRUX_CUDA(ctx, ctx->host_in.ensure(goff + std::max<size_t>(gbytes, 1)));
  char *din = ctx->host_in.as<char>();
  if (lde == N)
    KRUX_CUDA(ctx, cudaMemcpyAsync(din, expr, ebytes, cudaMemcpyHostToDevice, s));
  else
    KRUX_CUDA(ctx, cudaMemcpy2DAsync(din, (size_t)N * 4, expr, (size_t)lde * 4, (size_t)N * 4, T,
                                     cudaMemcpyHostToDevice, s));
  if (S > 0) {  // on the context's copy stream, while `stream` ranks
    if (!ctx->xs) {
      KRUX_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->xs, cudaStreamNonBlocking));
      KRUX_CUDA(ctx, cudaEventCreateWithFlags(&ctx->xev, cudaEventDisableTiming));
    }
    KRUX_CUDA(ctx, cudaEventRecord(ctx->xev, s));  // (after whatever `stream` holds)
    KRUX_CUDA(ctx, cudaStreamWaitEvent(ctx->xs, ctx->xev, 0));
    if (ldg == N)
      KRUX_CUDA(ctx, cudaMemcpyAsync(din + goff, geno, gbytes, cudaMemcpyHostToDevice, ctx->xs));
    else
      KRUX_CUDA(ctx, cudaMemcpy2DAsync(din + goff, (size_t)N, geno, (size_t)ldg, (size_t)N, S,
                                       cudaMemcpyHostToDevice, ctx->xs));
    KRUX_CUDA(ctx, cudaEventRecord(ctx->xev, ctx->xs));
  }
  const int64_t cap = std::max<int64_t>(opts->hit_capacity, 0);
  // outputs in page-locked memory mapped into the device's address space are
  // written by the compaction and finalisation kernels directly (no copy after
  // the launch); other outputs get a device list and three copies
  krux_hit *mh = nullptr;
  double *mH = nullptr, *mp = nullptr;
  if (cap > 0) {
    mh = static_cast<krux_hit *>(mapped_device_ptr(hits));
    mH = static_cast<double *>(mapped_device_ptr(hit_H));
    mp = static_cast<double *>(mapped_device_ptr(hit_p));
  }
  const bool direct = mh && mH && mp && ((uintptr_t)mh & 15u) == 0;
  const size_t hoff = 0, Hoff = (size_t)std::max<int64_t>(direct ? 0 : cap, 1) * sizeof(krux_hit);
  const size_t poff = Hoff + (size_t)std::max<int64_t>(direct ? 0 : cap, 1) * 8;
  KRUX_CUDA(ctx, ctx->host_out.ensure(poff + (size_t)std::max<int64_t>(direct ? 0 : cap, 1) * 8));
  char *dout = ctx->host_out.as<char>();
  krux_rankset *rs = nullptr;
  st = krux_rank(ctx, reinterpret_cast<const float *>(din), T, N, N, &rs, stream);
  if (st != KRUX_OK) {
    if (S > 0) cudaStreamSynchronize(ctx->xs);  // the caller's genotypes are read no more
    return st;
  }
  const float ms_rank = ctx->profiling ? ctx->prof.ms_rank : 0.f;
  if (S > 0) KRUX_CUDA(ctx, cudaStreamWaitEvent(s, ctx->xev, 0));  // the genotypes are in
  st = krux_scan(ctx, rs, reinterpret_cast<const int8_t *>(din + goff), S, N, opts,
                 direct ? mh : reinterpret_cast<krux_hit *>(dout + hoff),
                 direct ? mH : reinterpret_cast<double *>(dout + Hoff),
                 direct ? mp : reinterpret_cast<double *>(dout + poff), n_hits, stream);
  krux_rankset_free(ctx, rs);
  if (st != KRUX_OK && st != KRUX_EOVERFLOW) {
    cudaStreamSynchronize(s);  // (and with it the genotypes' copy it waited for)
    return st;
  }
  if (ctx->profiling) {
    ctx->prof.ms_rank = ms_rank;
    ctx->prof.launches += 2;  // the rank transform's two kernels
  }
  const int64_t k = direct ? 0 : std::min<int64_t>(*n_hits, cap);
  if (k > 0) {
    KRUX_CUDA(ctx, cudaMemcpyAsync(hits, dout + hoff, (size_t)k * sizeof(krux_hit),
                                   cudaMemcpyDeviceToHost, s));
    KRUX_CUDA(ctx, cudaMemcpyAsync(hit_H, dout + Hoff, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    KRUX_CUDA(ctx, cudaMemcpyAsync(hit_p, dout + poff, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
  }
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  return st;
}

extern "C" krux_status krux_scan_cis(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                                     int64_t S, int64_t ldg, const int64_t *snp_pos,
                                     const int64_t *trait_pos, int64_t window,
                                     const krux_opts *opts, krux_hit *hits, double *hit_H,
                                     double *hit_p, int64_t *n_hits, void *stream) {
  krux_status st = check_scan_args(ctx, rs, geno, S, ldg, opts, hits, hit_H, hit_p, n_hits);
  if (st != KRUX_OK) return st;
  *n_hits = 0;
  if (opts->dense_H || opts->dense_p)
    return fail(ctx, KRUX_EINVAL, "dense output is not available with a cis window");
  if (window < 0 || (S > 0 && !snp_pos) || !trait_pos)
    return fail(ctx, KRUX_EINVAL, "cis scan needs window >= 0 and both coordinate arrays");
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  CallPlan cp;
  cp.multi = (opts->flags & KRUX_FLAG_MULTIALLELIC) != 0;
  cp.cis.on = true;
  cp.cis.snp_pos = snp_pos;
  cp.cis.trait_pos = trait_pos;
  cp.cis.window = window;
  cp.cis.h_snp.resize((size_t)S);
  cp.cis.h_trait.resize((size_t)rs->T);
  if (S > 0)
    KRUX_CUDA(ctx, cudaMemcpyAsync(cp.cis.h_snp.data(), snp_pos, (size_t)S * 8,
                                   cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(cp.cis.h_trait.data(), trait_pos, (size_t)rs->T * 8,
                                 cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  if (!std::is_sorted(cp.cis.h_snp.begin(), cp.cis.h_snp.end()) ||
      !std::is_sorted(cp.cis.h_trait.begin(), cp.cis.h_trait.end()))
    return fail(ctx, KRUX_EINVAL, "cis coordinates must be nondecreasing");
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    ctx->prof.pairs = (int64_t)rs->T * (e - b);
  }
  KRUX_CUDA(ctx, ctx->aux.ensure((size_t)std::max<int64_t>(opts->hit_capacity, 1) * sizeof(HitAux)));
  cp.slots.push_back(OutSlot{hits, hit_H, hit_p, opts->hit_capacity, ctx->aux.as<HitAux>()});
  KRUX_CUDA(ctx, ctx->dlist.ensure((size_t)std::max<int64_t>(e - b, 1) * 8));
  st = plan_groups(ctx, cp, rs, geno, ldg, b, e, nullptr, 1, 0, nullptr, nullptr, nullptr, s);
  if (st != KRUX_OK) return st;
  st = materialise(ctx, cp, s);
  if (st != KRUX_OK) return st;
  std::vector<unsigned long long> counts;
  st = run_fused(ctx, cp, opts, s, counts);
  if (st != KRUX_OK) return st;
  *n_hits = (int64_t)counts[0];
  if (*n_hits > opts->hit_capacity)
    return fail(ctx, KRUX_EOVERFLOW, "%lld hits exceed capacity %lld", (long long)*n_hits,
                (long long)opts->hit_capacity);
  return KRUX_OK;
}

extern "C" krux_status krux_scan_parametric(krux_ctx *ctx, const float *expr, int T, int N,
                                            int64_t ld, const int8_t *geno, int64_t S,
                                            int64_t ldg, int model, const krux_opts *opts,
                                            krux_hit *hits, double *hit_stat, double *hit_p,
                                            int64_t *n_hits, void *stream) {
  if (!ctx) return KRUX_EINVAL;
  if (!n_hits) return fail(ctx, KRUX_EINVAL, "n_hits is NULL");
  *n_hits = 0;
  krux_status st = check_opts(ctx, opts);
  if (st != KRUX_OK) return st;
  if (opts->flags != 0 || opts->dense_H)
    return fail(ctx, KRUX_EINVAL, "parametric scans take no flags and no dense output");
  if (model != 0 && model != 1) return fail(ctx, KRUX_EINVAL, "model must be 0 (ANOVA) or 1 (linear)");
  if (!expr || T < 1 || N < 4 || N > kMaxN || ld < N)
    return fail(ctx, KRUX_EINVAL, "need expr, T >= 1, 4 <= N <= %d and ld >= N", kMaxN);
  if (S < 0 || (S > 0 && (!geno || ldg < N)) || S >= ((int64_t)1 << 31))
    return fail(ctx, KRUX_EINVAL, "bad genotype matrix");
  if (opts->hit_capacity > 0 && (!hits || !hit_stat || !hit_p))
    return fail(ctx, KRUX_EINVAL, "hit outputs are NULL");
  if (((uintptr_t)hits & 15u) != 0) return fail(ctx, KRUX_EINVAL, "hits must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  if (b < 0 || e > S || b > e) return fail(ctx, KRUX_EINVAL, "bad SNP slice");
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    ctx->prof.pairs = (int64_t)T * (e - b);
  }
  // the standardised values in the layout of a rank set
  krux_rankset rs;
  rs.T = T;
  rs.N = N;
  rs.Np = round_up(N, 16);
  rs.rows_pad = round_up(T, kTileM);
  rs.n_ttiles = rs.rows_pad / kTileM;
  rs.has_nan = false;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t oA = take((size_t)rs.rows_pad * rs.Np * 2), oTau = take((size_t)rs.rows_pad * 4),
               oCf = take((size_t)rs.rows_pad * 8), oNc = take((size_t)rs.rows_pad * 2),
               oNi = take((size_t)T * N * 2), oTile = take((size_t)rs.n_ttiles * 4),
               oMean = take((size_t)T * 8), oSd = take((size_t)T * 8);
  KRUX_CUDA(ctx, ctx->param.ensure(off));
  char *pb = ctx->param.as<char>();
  KRUX_CUDA(ctx, cudaMemsetAsync(pb, 0, off, s));
  rs.dev = RankDev{};
  rs.dev.A = reinterpret_cast<__half *>(pb + oA);
  rs.dev.tau = reinterpret_cast<float *>(pb + oTau);
  rs.dev.cfac = reinterpret_cast<double *>(pb + oCf);
  rs.dev.nan_cnt = reinterpret_cast<uint16_t *>(pb + oNc);
  rs.dev.nan_idx = reinterpret_cast<uint16_t *>(pb + oNi);
  rs.dev.tile_nan = reinterpret_cast<uint32_t *>(pb + oTile);
  double *mean = reinterpret_cast<double *>(pb + oMean);
  double *sd = reinterpret_cast<double *>(pb + oSd);
  KRUX_CUDA(ctx, ctx->status.ensure(64));
  KRUX_CUDA(ctx, cudaMemsetAsync(ctx->status.p, 0, 64, s));
  ev_record(ctx, 0, s);
  KRUX_CUDA(ctx, launch_standardize(expr, T, N, ld, rs.Np, rs.dev.A, mean, sd, rs.dev.tau,
                                    rs.dev.cfac, rs.dev.nan_cnt, ctx->status.as<unsigned int>(), s));
  KRUX_CUDA(ctx, launch_pad_traits(T, rs.rows_pad, rs.dev.tau, rs.dev.cfac, rs.dev.nan_cnt, s));
  ev_record(ctx, 1, s);
  unsigned int hst = 0;
  KRUX_CUDA(ctx, cudaMemcpyAsync(&hst, ctx->status.p, 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  if (hst & kDevBadCode) return fail(ctx, KRUX_EINVAL, "parametric scans take expression without NaN");
  // bounds of the fused test
  CallPlan cp;
  cp.param.model = model;
  const double K = (double)N;
  if (model == 0) {
    for (int df = 1; df <= 2; ++df) {
      const double fc = param_f_crit(opts->pthresh, df, K - 1.0 - df);
      const double tau = (K - 1.0) * fc * df / (K - 1.0 - df + fc * df);
      (df == 1 ? cp.param.h1 : cp.param.h2) = tau;
    }
  } else {
    const double tc = param_t_crit(opts->pthresh, K - 2.0);
    const double rc2 = tc * tc / (K - 2.0 + tc * tc);
    cp.param.rl = 1.0 / ((K - 1.0) * rc2);
  }
  cp.param.expr = expr;
  cp.param.ld = ld;
  cp.param.mean = mean;
  cp.param.out = hits;
  cp.param.out_stat = hit_stat;
  cp.param.out_p = hit_p;
  cp.param.out_capacity = opts->hit_capacity;
  // provisional hits: the caller's capacity plus room for the band
  const int64_t prov = opts->hit_capacity + ((int64_t)1 << 20);
  KRUX_CUDA(ctx, ctx->paramOut.ensure((size_t)prov * (16 + 8 + 8)));
  krux_hit *ph = ctx->paramOut.as<krux_hit>();
  double *pstat = reinterpret_cast<double *>(ctx->paramOut.as<char>() + (size_t)prov * 16);
  double *pp = pstat + prov;
  KRUX_CUDA(ctx, ctx->aux.ensure((size_t)prov * sizeof(HitAux)));
  cp.slots.push_back(OutSlot{ph, pstat, pp, prov, ctx->aux.as<HitAux>()});
  st = plan_groups(ctx, cp, &rs, geno, ldg, b, e, nullptr, 1, 0, nullptr, nullptr, nullptr, s);
  if (st != KRUX_OK) return st;
  if (!cp.bucket_jobs.empty())
    return fail(ctx, KRUX_EUNSUPPORTED, "parametric scans take complete genotypes (no -1 codes)");
  st = materialise(ctx, cp, s);
  if (st != KRUX_OK) return st;
  std::vector<unsigned long long> counts;
  st = run_fused(ctx, cp, opts, s, counts);
  if (st != KRUX_OK) return st;
  unsigned long long n_final = 0;
  KRUX_CUDA(ctx, cudaMemcpyAsync(&n_final, ctx->counters.as<unsigned long long>() + 2, 8,
                                 cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  if (ctx->profiling) ctx->prof.ms_rank = ev_ms(ctx, 0, 1);
  if ((int64_t)counts[0] > prov) {
    *n_hits = (int64_t)counts[0];
    return fail(ctx, KRUX_EOVERFLOW,
                "%lld provisional hits exceed the work list; n_hits is an upper bound",
                (long long)counts[0]);
  }
  *n_hits = (int64_t)n_final;
  if (*n_hits > opts->hit_capacity)
    return fail(ctx, KRUX_EOVERFLOW, "%lld hits exceed capacity %lld", (long long)*n_hits,
                (long long)opts->hit_capacity);
  return KRUX_OK;
}

extern "C" krux_status krux_scan_grouped(krux_ctx *ctx, krux_cohort *cohorts, int n_cohorts,
                                         const krux_opts *opts, void *stream) {
  if (!ctx) return KRUX_EINVAL;
  krux_status st = check_opts(ctx, opts);
  if (st != KRUX_OK) return st;
  if (n_cohorts < 0 || (n_cohorts > 0 && !cohorts)) return fail(ctx, KRUX_EINVAL, "bad cohort list");
  if (opts->dense_H) return fail(ctx, KRUX_EINVAL, "dense output is not available for grouped scans");
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t captot = 0;
  for (int c = 0; c < n_cohorts; ++c) {
    krux_cohort &k = cohorts[c];
    k.n_hits = 0;
    if (!k.rs || k.S < 0 || (k.S > 0 && (!k.geno || k.ldg < k.rs->N)) || k.hit_capacity < 0 ||
        (k.hit_capacity > 0 && (!k.hits || !k.hit_H || !k.hit_p)) || ((uintptr_t)k.hits & 15u) != 0)
      return fail(ctx, KRUX_EINVAL, "cohort %d: bad arguments", c);
    captot += std::max<int64_t>(k.hit_capacity, 1);
  }
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    for (int c = 0; c < n_cohorts; ++c) ctx->prof.pairs += (int64_t)cohorts[c].rs->T * cohorts[c].S;
  }
  KRUX_CUDA(ctx, ctx->aux.ensure((size_t)std::max<int64_t>(captot, 1) * sizeof(HitAux)));
  {
    int64_t snps = 1;
    for (int c = 0; c < n_cohorts; ++c) snps += cohorts[c].S;
    KRUX_CUDA(ctx, ctx->dlist.ensure((size_t)snps * 8));
  }
  CallPlan cp;
  cp.multi = (opts->flags & KRUX_FLAG_MULTIALLELIC) != 0;
  int64_t aoff = 0;
  for (int c = 0; c < n_cohorts; ++c) {
    krux_cohort &k = cohorts[c];
    cp.slots.push_back(OutSlot{k.hits, k.hit_H, k.hit_p, k.hit_capacity, ctx->aux.as<HitAux>() + aoff});
    aoff += std::max<int64_t>(k.hit_capacity, 1);
    st = plan_groups(ctx, cp, k.rs, k.geno, k.ldg, 0, k.S, nullptr, 1, c, nullptr, nullptr, nullptr, s);
    if (st != KRUX_OK) return st;
  }
  st = materialise(ctx, cp, s);
  if (st != KRUX_OK) return st;
  // Cohorts whose every group can take the plain scan form run in one launch of
  // that form, the others in one launch of the general form (one launch holds one
  // form); each cohort's groups stay in one launch, so its hit list has one writer.
  std::vector<char> plain(n_cohorts, cp.multi ? 0 : 1);
  for (const ScanGroupIn &g : cp.groups)
    if (g.nan_cnt || g.bucket >= 0 || !plain_form_fits(ctx, g.rs->Np)) plain[g.out_slot] = 0;
  CallPlan parts[2];
  for (int k = 0; k < 2; ++k) {
    parts[k] = cp;
    parts[k].groups.clear();
  }
  for (const ScanGroupIn &g : cp.groups) parts[plain[g.out_slot] ? 0 : 1].groups.push_back(g);
  std::vector<unsigned long long> total(n_cohorts, 0ull);
  float ms_scan = 0.f;
  int launches = 0;
  for (int k = 0; k < 2; ++k) {
    if (parts[k].groups.empty()) continue;
    std::vector<unsigned long long> counts;
    st = run_fused(ctx, parts[k], opts, s, counts);
    if (st != KRUX_OK) return st;
    for (const ScanGroupIn &g : parts[k].groups) total[g.out_slot] = counts[g.out_slot];
    ms_scan += ctx->prof.ms_scan;
    launches = ctx->prof.launches;
  }
  if (ctx->profiling) {
    ctx->prof.ms_scan = ms_scan;
    ctx->prof.launches = launches;
  }
  bool over = false;
  for (int c = 0; c < n_cohorts; ++c) {
    cohorts[c].n_hits = (int64_t)total[c];
    over |= cohorts[c].n_hits > cohorts[c].hit_capacity;
  }
  if (over) return fail(ctx, KRUX_EOVERFLOW, "a cohort's hits exceed its capacity");
  return KRUX_OK;
}

extern "C" krux_status krux_scan_plain(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                                       int64_t S, int64_t ldg, const krux_opts *opts, krux_hit *hits,
                                       double *hit_H, double *hit_p, int64_t *n_hits, void *stream) {
  krux_status st = check_scan_args(ctx, rs, geno, S, ldg, opts, hits, hit_H, hit_p, n_hits);
  if (st != KRUX_OK) return st;
  if (opts->flags & KRUX_FLAG_MULTIALLELIC)
    return fail(ctx, KRUX_EUNSUPPORTED, "this form takes biallelic markers (codes 0, 1, 2) only");
  *n_hits = 0;
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  const int64_t n = e - b;
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    ctx->prof.pairs = (int64_t)rs->T * n;
  }
  if (n == 0) return KRUX_OK;
  std::vector<Bucket> buckets;
  std::vector<int64_t> complete;
  bool bad = false;
  st = find_missing(ctx, geno, ldg, rs->N, b, n, s, buckets, complete, bad, 2);
  if (st != KRUX_OK) return st;
  if (bad) return fail(ctx, KRUX_EINVAL, "genotype code outside {-1,0,1,2}");
  if (!buckets.empty())
    return fail(ctx, KRUX_EUNSUPPORTED, "the plain form takes complete genotypes only");
  if (!ctx->blas) ctx->blas = plain_handle_create();
  if (!ctx->blas) return fail(ctx, KRUX_ECUDA, "cublasCreate failed");
  const double h1 = h_df1(opts->pthresh), h2 = h_df2(opts->pthresh);
  const int64_t nch = (n + kChunkSnps - 1) / kChunkSnps;
  KRUX_CUDA(ctx, ctx->B.ensure((size_t)nch * kChunkRows * rs->Np * 2));
  KRUX_CUDA(ctx, ctx->meta.ensure((size_t)nch * sizeof(ChunkMeta)));
  KRUX_CUDA(ctx, ctx->aux.ensure((size_t)std::max<int64_t>(opts->hit_capacity, 1) * sizeof(HitAux)));
  KRUX_CUDA(ctx, ctx->counters.ensure(64));
  KRUX_CUDA(ctx, ctx->status.ensure(64));
  KRUX_CUDA(ctx, cudaMemsetAsync(ctx->counters.p, 0, 64, s));
  KRUX_CUDA(ctx, cudaMemsetAsync(ctx->status.p, 0, 64, s));
  ev_record(ctx, 2, s);
  KRUX_CUDA(ctx, launch_pack2(geno, ldg, rs->N, rs->Np, nullptr, b, n, 0, h1, h2, 0, 0,
                              ctx->B.as<__half>(), ctx->meta.as<ChunkMeta>(), nullptr,
                              ctx->status.as<unsigned int>(), s));
  ev_record(ctx, 3, s);
  // SNP slices whose T x 2*slice FP32 rank-sum matrix fits a 4 GiB buffer
  const int64_t budget = (int64_t)4 << 30;
  int64_t cs = std::max<int64_t>(1, budget / ((int64_t)rs->rows_pad * kChunkRows * 4));
  cs = std::min(cs, nch);
  KRUX_CUDA(ctx, ctx->gemm_out.ensure((size_t)rs->rows_pad * cs * kChunkRows * 4));
  const float margin = (float)(opts->recheck_margin > 0 ? opts->recheck_margin : 1e-4);
  int launches = 1;
  for (int64_t c0 = 0; c0 < nch; c0 += cs) {
    const int64_t cn = std::min(cs, nch - c0);
    const int rowsB = (int)(cn * kChunkRows);
    KRUX_CUDA(ctx, plain_gemm(ctx->blas, rs->dev.A, rs->rows_pad, rs->Np,
                              ctx->B.as<__half>() + (size_t)c0 * kChunkRows * rs->Np, rowsB,
                              ctx->gemm_out.as<float>(), s));
    const int n_slots = (int)std::min<int64_t>(cn * kChunkSnps, n - c0 * kChunkSnps);
    KRUX_CUDA(ctx, launch_plain_epilogue2(
                       ctx->gemm_out.as<float>(), rowsB, rs->T, n_slots, ctx->meta.as<ChunkMeta>() + c0,
                       rs->dev.tau, rs->dev.cfac, rs->has_nan ? rs->dev.nan_cnt : nullptr,
                       rs->dev.nan_idx, rs->N, geno, ldg, margin, opts->pthresh, (float)h1, (float)h2,
                       hits, ctx->aux.as<HitAux>(), ctx->counters.as<unsigned long long>(),
                       opts->hit_capacity, opts->dense_H, opts->dense_p, n, b, s));
    launches += 2;
  }
  ev_record(ctx, 4, s);
  unsigned long long cnt = 0;
  unsigned int hst = 0;
  KRUX_CUDA(ctx, cudaMemcpyAsync(&cnt, ctx->counters.p, 8, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaMemcpyAsync(&hst, ctx->status.p, 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  if (hst & kDevBadCode) return fail(ctx, KRUX_EINVAL, "genotype code outside {-1,0,1,2}");
  const double *cf = rs->dev.cfac;
  KRUX_CUDA(ctx, ctx->cfacptr.ensure(sizeof(double *)));
  KRUX_CUDA(ctx, cudaMemcpyAsync(ctx->cfacptr.p, &cf, sizeof(double *), cudaMemcpyHostToDevice, s));
  ev_record(ctx, 5, s);
  const int64_t nst = std::min<int64_t>((int64_t)cnt, opts->hit_capacity);
  if (nst > 0)
    KRUX_CUDA(ctx, launch_finalize(hits, ctx->aux.as<HitAux>(), nst, ctx->cfacptr.as<const double *>(),
                                   hit_H, hit_p, s, nullptr, 0, 0.0, 1.0, opts->pthresh));
  ev_record(ctx, 6, s);
  if (ctx->profiling) {
    KRUX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->prof.ms_pack = ev_ms(ctx, 2, 3);
    ctx->prof.ms_scan = ev_ms(ctx, 3, 4);
    ctx->prof.ms_finalize = ev_ms(ctx, 5, 6);
    ctx->prof.launches = launches + (nst > 0 ? 1 : 0) + 1;
  }
  *n_hits = (int64_t)cnt;
  if (*n_hits > opts->hit_capacity)
    return fail(ctx, KRUX_EOVERFLOW, "%lld hits exceed capacity %lld", (long long)*n_hits,
                (long long)opts->hit_capacity);
  return KRUX_OK;
}

// Plans a permutation batch: the 1 + P stacked rank matrices as one group (the
// stacking itself is queued by enqueue_fused).
static krux_status plan_permute(krux_ctx *ctx, CallPlan &cp, const krux_rankset *rs, const int8_t *geno,
                         int64_t S, int64_t ldg, const int32_t *perms, int P,
                         const krux_opts *opts, double *minp, krux_hit *hits, double *hit_H,
                         double *hit_p, uint64_t *fdr_hist, int fdr_bins, double fdr_bin_width,
                         cudaStream_t s) {
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  const size_t one = (size_t)rs->rows_pad * rs->Np;
  KRUX_CUDA(ctx, ctx->permA.ensure(one * 2 * (size_t)(1 + P)));
  // [P][rows_pad] FP64 keys, then the plain form's [P][rows_pad][2] 64-bit bounds and
  // [P][rows_pad][2] 64-bit seed records
  KRUX_CUDA(ctx, ctx->minpkey.ensure((size_t)P * rs->rows_pad * 40));
  KRUX_CUDA(ctx, ctx->aux.ensure((size_t)std::max<int64_t>(opts->hit_capacity, 1) * sizeof(HitAux)));
  cp.slots.push_back(OutSlot{hits, hit_H, hit_p, opts->hit_capacity, ctx->aux.as<HitAux>()});
  cp.fdr_hist = reinterpret_cast<unsigned long long *>(fdr_hist);
  cp.fdr_rows = 1 + P;
  cp.fdr_bins = fdr_bins;
  cp.fdr_l0 = -std::log10(opts->pthresh);
  cp.fdr_w = fdr_bin_width;
  cp.perm.on = true;
  cp.perm.rs = rs;
  cp.perm.perms = perms;
  cp.perm.P = P;
  cp.perm.stack = ctx->permA.as<__half>();
  cp.perm.minp = minp;
  krux_status st = plan_groups(ctx, cp, rs, geno, ldg, b, e, cp.perm.stack, 1 + P, 0, nullptr,
                               nullptr, ctx->minpkey.as<double>(), s);
  if (st != KRUX_OK) return st;
  for (auto &g : cp.groups)
    if (g.minp_key) {
      g.minp_bound = reinterpret_cast<unsigned long long *>(ctx->minpkey.as<double>() +
                                                            (size_t)P * rs->rows_pad);
      g.minp_seed = reinterpret_cast<unsigned long long *>(ctx->minpkey.as<double>() +
                                                           (size_t)3 * P * rs->rows_pad);
    }
  if (rs->has_nan) {
    const size_t lst = (size_t)rs->T * rs->N;
    const size_t inv_off = (lst * 2 * (size_t)(1 + P) + 255) / 256 * 256;
    KRUX_CUDA(ctx, ctx->permNan.ensure(inv_off + (size_t)P * rs->N * 4));
    cp.perm.lists = ctx->permNan.as<uint16_t>();
    cp.perm.inv = reinterpret_cast<int32_t *>(ctx->permNan.as<char>() + inv_off);
    for (auto &g : cp.groups) {
      g.nan_idx = cp.perm.lists;
      g.nan_ag_stride = (int64_t)lst;
    }
  }
  return materialise(ctx, cp, s);
}

extern "C" krux_status krux_permute(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                                    int64_t S, int64_t ldg, const int32_t *perms, int P,
                                    const krux_opts *opts, double *minp, krux_hit *hits,
                                    double *hit_H, double *hit_p, int64_t *n_hits,
                                    uint64_t *fdr_hist, int fdr_bins, double fdr_bin_width,
                                    void *stream) {
  krux_status st = check_scan_args(ctx, rs, geno, S, ldg, opts, hits, hit_H, hit_p, n_hits);
  if (st != KRUX_OK) return st;
  if (opts->flags & KRUX_FLAG_MULTIALLELIC)
    return fail(ctx, KRUX_EUNSUPPORTED, "this form takes biallelic markers (codes 0, 1, 2) only");
  *n_hits = 0;
  if (P < 1 || !perms || !minp) return fail(ctx, KRUX_EINVAL, "need P >= 1, perms and minp");
  if (opts->dense_H) return fail(ctx, KRUX_EINVAL, "dense output is not available with permutations");
  if (fdr_hist && (fdr_bins < 1 || !(fdr_bin_width > 0.0)))
    return fail(ctx, KRUX_EINVAL, "FDR histogram needs fdr_bins >= 1 and fdr_bin_width > 0");
  cudaStream_t s = (cudaStream_t)stream;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  const int N = rs->N;
  // every row must be a permutation of 0..N-1 (checked on the host before any gather)
  std::vector<int32_t> hp((size_t)P * N);
  KRUX_CUDA(ctx, cudaMemcpyAsync(hp.data(), perms, hp.size() * 4, cudaMemcpyDeviceToHost, s));
  KRUX_CUDA(ctx, cudaStreamSynchronize(s));
  for (int q = 0; q < P; ++q) {
    std::vector<char> seen(N, 0);
    for (int k = 0; k < N; ++k) {
      const int32_t v = hp[(size_t)q * N + k];
      if (v < 0 || v >= N || seen[v]) return fail(ctx, KRUX_EINVAL, "perms row %d is not a permutation", q);
      seen[v] = 1;
    }
  }
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  if (ctx->profiling) {
    ctx->prof = krux_profile{};
    ctx->prof.pairs = (int64_t)rs->T * (e - b) * (1 + P);
  }
  CallPlan cp;
  st = plan_permute(ctx, cp, rs, geno, S, ldg, perms, P, opts, minp, hits, hit_H, hit_p, fdr_hist,
                    fdr_bins, fdr_bin_width, s);
  if (st != KRUX_OK) return st;
  // the main launch is prepared first (it sizes every buffer the two launches
  // share), the seed pass into the second table set, then both are enqueued back
  // to back with no host synchronisation between them
  CallPlan seed;
  FusedLaunch fm, fs;
  st = prepare_fused(ctx, cp, opts, fm, s, 0);
  if (st != KRUX_OK) return st;
  const bool with_seed = make_seed_plan(cp, seed, fm.p.fast != 0);
  if (with_seed) {
    st = prepare_fused(ctx, seed, opts, fs, s, 1);
    if (st != KRUX_OK) return st;
    KRUX_CUDA(ctx, scan_set_smem(std::max(fs.smem, fm.smem)));
    st = enqueue_fused(ctx, seed, fs, s);
    if (st != KRUX_OK) return st;
    if (ctx->profiling) ctx->prof.launches += fused_launches(seed, fs);
    cp.perm.pre_done = true;
  }
  st = enqueue_fused(ctx, cp, fm, s);
  if (st != KRUX_OK) return st;
  std::vector<unsigned long long> counts;
  st = finish_fused(ctx, cp, fm, s, counts);
  if (st != KRUX_OK) return st;
  *n_hits = (int64_t)counts[0];
  if (*n_hits > opts->hit_capacity)
    return fail(ctx, KRUX_EOVERFLOW, "%lld hits exceed capacity %lld", (long long)*n_hits,
                (long long)opts->hit_capacity);
  return KRUX_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs: one call's stream work (permutation stacking, packing, the fused
// scan, compaction, FP64 finalisation, min-p conversion) captured once and
// replayed.  The graph owns a private workspace (its own context buffers), so
// later calls on the caller's context cannot move memory the graph uses.
struct krux_graph {
  krux_ctx *w = nullptr;           // private workspace context
  CallPlan cp;
  FusedLaunch fl;
  bool with_seed = false;          // a permutation batch's seed pass runs first
  CallPlan seed_cp;
  FusedLaunch seed_fl;
  krux_opts opts{};
  cudaStream_t cs = nullptr;       // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long *host = nullptr;  // pinned: [nslots] totals, then 2 status words
  cudaStream_t last = nullptr;     // stream of the last launch
  bool launched = false;
};

namespace {

krux_ctx *workspace_clone(const krux_ctx *src) {
  krux_ctx *w = new krux_ctx();
  w->device = src->device;
  w->sm_count = src->sm_count;
  w->cc_major = src->cc_major;
  w->cc_minor = src->cc_minor;
  w->wait_limit = src->wait_limit;
  w->tune_layout = src->tune_layout;
  w->tune_nc = src->tune_nc;
  w->tune_nA = src->tune_nA;
  w->tune_ka = src->tune_ka;
  w->tuned = src->tuned;
  w->encode = src->encode;
  w->profiling = false;
  return w;
}

void graph_free(krux_graph *g) {
  if (!g) return;
  if (g->w) cudaSetDevice(g->w->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cs) cudaStreamDestroy(g->cs);
  if (g->host) cudaFreeHost(g->host);
  if (g->w) krux_destroy(g->w);
  delete g;
}

// Copies the workspace's error text to the caller's context and frees the graph.
krux_status graph_fail(krux_ctx *ctx, krux_graph *g, krux_status st) {
  if (g && g->w && !g->w->err.empty()) ctx->err = g->w->err;
  graph_free(g);
  return st;
}

// Prepares, then captures enqueue_fused plus the read-back of the counts into
// pinned host memory.
krux_status graph_capture(krux_ctx *ctx, krux_graph *g) {
  krux_ctx *w = g->w;
  if (!g->cp.bucket_jobs.empty() || !g->cp.lists.empty())
    return fail(ctx, KRUX_EUNSUPPORTED, "graphs take complete genotypes (no -1 codes)");
  krux_status st = prepare_fused(w, g->cp, &g->opts, g->fl, g->cs);
  if (st != KRUX_OK) return st;
  if (g->with_seed) g->with_seed = make_seed_plan(g->cp, g->seed_cp, g->fl.p.fast != 0);
  if (g->with_seed) {
    st = prepare_fused(w, g->seed_cp, &g->opts, g->seed_fl, g->cs, 1);
    if (st != KRUX_OK) return st;
    KRUX_CUDA(w, scan_set_smem(std::max(g->seed_fl.smem, g->fl.smem)));
    g->cp.perm.pre_done = true;
  }
  const int nslots = g->fl.nslots;
  KRUX_CUDA(w, cudaHostAlloc(reinterpret_cast<void **>(&g->host), (size_t)(nslots + 1) * 8,
                             cudaHostAllocDefault));
  std::memset(g->host, 0, (size_t)(nslots + 1) * 8);
  KRUX_CUDA(w, cudaStreamSynchronize(g->cs));
  KRUX_CUDA(w, cudaStreamBeginCapture(g->cs, cudaStreamCaptureModeThreadLocal));
  if (g->with_seed) st = enqueue_fused(w, g->seed_cp, g->seed_fl, g->cs);
  if (st == KRUX_OK) st = enqueue_fused(w, g->cp, g->fl, g->cs);
  if (st == KRUX_OK && cudaMemcpyAsync(g->host, w->counters.as<unsigned long long>() + nslots,
                                       (size_t)nslots * 8, cudaMemcpyDeviceToHost, g->cs) != cudaSuccess)
    st = fail(w, KRUX_ECUDA, "capture of the count read-back failed");
  if (st == KRUX_OK && cudaMemcpyAsync(g->host + nslots, w->status.p, 8, cudaMemcpyDeviceToHost,
                                       g->cs) != cudaSuccess)
    st = fail(w, KRUX_ECUDA, "capture of the status read-back failed");
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(g->cs, &graph);
  if (st != KRUX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ec != cudaSuccess)
    return fail(w, KRUX_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ec));
  g->graph = graph;
  KRUX_CUDA(w, cudaGraphInstantiate(&g->exec, g->graph, 0));
  return KRUX_OK;
}

krux_status graph_begin(krux_ctx *ctx, krux_graph **out, krux_graph *&g) {
  *out = nullptr;
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  g = new krux_graph();
  g->w = workspace_clone(ctx);
  if (cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking) != cudaSuccess) {
    graph_free(g);
    g = nullptr;
    return fail(ctx, KRUX_ECUDA, "cudaStreamCreateWithFlags failed");
  }
  return KRUX_OK;
}

}  // namespace

extern "C" krux_status krux_graph_scan(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                                       int64_t S, int64_t ldg, const krux_opts *opts,
                                       krux_hit *hits, double *hit_H, double *hit_p,
                                       krux_graph **out) {
  if (!out) return KRUX_EINVAL;
  int64_t dummy = 0;
  krux_status st = check_scan_args(ctx, rs, geno, S, ldg, opts, hits, hit_H, hit_p, &dummy);
  if (st != KRUX_OK) return st;
  krux_graph *g = nullptr;
  st = graph_begin(ctx, out, g);
  if (st != KRUX_OK) return st;
  g->opts = *opts;
  g->cp.multi = (opts->flags & KRUX_FLAG_MULTIALLELIC) != 0;
  krux_ctx *w = g->w;
  const int64_t b = opts->snp_begin, e = opts->snp_end > 0 ? opts->snp_end : S;
  if (w->aux.ensure((size_t)std::max<int64_t>(opts->hit_capacity, 1) * sizeof(HitAux)) != cudaSuccess)
    return graph_fail(ctx, g, fail(ctx, KRUX_ENOMEM, "graph workspace"));
  g->cp.slots.push_back(OutSlot{hits, hit_H, hit_p, opts->hit_capacity, w->aux.as<HitAux>()});
  st = plan_groups(w, g->cp, rs, geno, ldg, b, e, nullptr, 1, 0, opts->dense_H, opts->dense_p,
                   nullptr, g->cs);
  if (st == KRUX_OK) st = materialise(w, g->cp, g->cs);
  if (st == KRUX_OK) st = graph_capture(ctx, g);
  if (st != KRUX_OK) return graph_fail(ctx, g, st);
  *out = g;
  return KRUX_OK;
}

extern "C" krux_status krux_graph_permute(krux_ctx *ctx, const krux_rankset *rs,
                                          const int8_t *geno, int64_t S, int64_t ldg,
                                          const int32_t *perms, int P, const krux_opts *opts,
                                          double *minp, krux_hit *hits, double *hit_H,
                                          double *hit_p, uint64_t *fdr_hist, int fdr_bins,
                                          double fdr_bin_width, krux_graph **out) {
  if (!out) return KRUX_EINVAL;
  int64_t dummy = 0;
  krux_status st = check_scan_args(ctx, rs, geno, S, ldg, opts, hits, hit_H, hit_p, &dummy);
  if (st != KRUX_OK) return st;
  if (opts->flags & KRUX_FLAG_MULTIALLELIC)
    return fail(ctx, KRUX_EUNSUPPORTED, "this form takes biallelic markers (codes 0, 1, 2) only");
  if (P < 1 || !perms || !minp) return fail(ctx, KRUX_EINVAL, "need P >= 1, perms and minp");
  if (opts->dense_H) return fail(ctx, KRUX_EINVAL, "dense output is not available with permutations");
  if (fdr_hist && (fdr_bins < 1 || !(fdr_bin_width > 0.0)))
    return fail(ctx, KRUX_EINVAL, "FDR histogram needs fdr_bins >= 1 and fdr_bin_width > 0");
  krux_graph *g = nullptr;
  st = graph_begin(ctx, out, g);
  if (st != KRUX_OK) return st;
  g->opts = *opts;
  st = plan_permute(g->w, g->cp, rs, geno, S, ldg, perms, P, opts, minp, hits, hit_H, hit_p,
                    fdr_hist, fdr_bins, fdr_bin_width, g->cs);
  if (st == KRUX_OK) g->with_seed = true;  // the plan is made once the main launch is prepared
  if (st == KRUX_OK) st = graph_capture(ctx, g);
  if (st != KRUX_OK) return graph_fail(ctx, g, st);
  *out = g;
  return KRUX_OK;
}

extern "C" krux_status krux_graph_grouped(krux_ctx *ctx, const krux_cohort *cohorts, int n_cohorts,
                                          const krux_opts *opts, krux_graph **out) {
  if (!ctx || !out) return KRUX_EINVAL;
  krux_status st = check_opts(ctx, opts);
  if (st != KRUX_OK) return st;
  if (n_cohorts < 1 || !cohorts) return fail(ctx, KRUX_EINVAL, "bad cohort list");
  if (opts->dense_H) return fail(ctx, KRUX_EINVAL, "dense output is not available for grouped scans");
  int64_t captot = 0;
  for (int c = 0; c < n_cohorts; ++c) {
    const krux_cohort &k = cohorts[c];
    if (!k.rs || k.S < 0 || (k.S > 0 && (!k.geno || k.ldg < k.rs->N)) || k.hit_capacity < 0 ||
        (k.hit_capacity > 0 && (!k.hits || !k.hit_H || !k.hit_p)) || ((uintptr_t)k.hits & 15u) != 0)
      return fail(ctx, KRUX_EINVAL, "cohort %d: bad arguments", c);
    captot += std::max<int64_t>(k.hit_capacity, 1);
  }
  krux_graph *g = nullptr;
  st = graph_begin(ctx, out, g);
  if (st != KRUX_OK) return st;
  g->opts = *opts;
  g->cp.multi = (opts->flags & KRUX_FLAG_MULTIALLELIC) != 0;
  krux_ctx *w = g->w;
  if (w->aux.ensure((size_t)std::max<int64_t>(captot, 1) * sizeof(HitAux)) != cudaSuccess)
    return graph_fail(ctx, g, fail(ctx, KRUX_ENOMEM, "graph workspace"));
  int64_t aoff = 0;
  for (int c = 0; c < n_cohorts && st == KRUX_OK; ++c) {
    const krux_cohort &k = cohorts[c];
    g->cp.slots.push_back(
        OutSlot{k.hits, k.hit_H, k.hit_p, k.hit_capacity, w->aux.as<HitAux>() + aoff});
    aoff += std::max<int64_t>(k.hit_capacity, 1);
    st = plan_groups(w, g->cp, k.rs, k.geno, k.ldg, 0, k.S, nullptr, 1, c, nullptr, nullptr,
                     nullptr, g->cs);
  }
  if (st == KRUX_OK) st = materialise(w, g->cp, g->cs);
  if (st == KRUX_OK) st = graph_capture(ctx, g);
  if (st != KRUX_OK) return graph_fail(ctx, g, st);
  *out = g;
  return KRUX_OK;
}

extern "C" krux_status krux_graph_launch(krux_graph *g, void *stream) {
  if (!g || !g->exec) return KRUX_EINVAL;
  if (cudaSetDevice(g->w->device) != cudaSuccess) return KRUX_ECUDA;
  const cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(g->w, KRUX_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  g->last = (cudaStream_t)stream;
  g->launched = true;
  return KRUX_OK;
}

extern "C" krux_status krux_graph_wait(krux_graph *g, int64_t *n_hits, int n_lists) {
  if (!g || !g->launched) return KRUX_EINVAL;
  const int nslots = g->fl.nslots;
  if (n_lists < nslots || (nslots > 0 && !n_hits)) return KRUX_EINVAL;
  if (cudaSetDevice(g->w->device) != cudaSuccess) return KRUX_ECUDA;
  const cudaError_t e = cudaStreamSynchronize(g->last);
  if (e != cudaSuccess) return fail(g->w, KRUX_ECUDA, "%s", cudaGetErrorString(e));
  unsigned int hst[2];
  std::memcpy(hst, g->host + nslots, 8);
  bool over = false;
  for (int k = 0; k < nslots; ++k) {
    n_hits[k] = (int64_t)g->host[k];
    over |= n_hits[k] > g->cp.slots[k].capacity;
  }
  const krux_status st = device_status(g->w, hst);
  if (st != KRUX_OK) return st;
  if (hst[0] & kDevMissing)
    return fail(g->w, KRUX_EUNSUPPORTED, "a -1 genotype code appeared in a graph replay");
  if (over) return fail(g->w, KRUX_EOVERFLOW, "hits exceed a list's capacity");
  return KRUX_OK;
}

extern "C" const char *krux_graph_last_error(const krux_graph *g) {
  return g && g->w ? g->w->err.c_str() : "";
}

extern "C" void krux_graph_destroy(krux_graph *g) { graph_free(g); }

// ---------------------------------------------------------------------------
// Autotuner: times the fused scan of this rank set over a sample of the SNPs
// (the first 65,536) for every launch shape that fits, and keeps the fastest for
// the rank set's K width; later launches of that width use it unless a shape is
// set explicitly with krux_set_tuning.
extern "C" krux_status krux_autotune(krux_ctx *ctx, const krux_rankset *rs, const int8_t *geno,
                                     int64_t S, int64_t ldg, double pthresh, void *stream,
                                     int32_t *shape_out) {
  if (!ctx) return KRUX_EINVAL;
  if (!rs || !geno || S < 1 || ldg < rs->N || !(pthresh > 0.0 && pthresh < 1.0))
    return fail(ctx, KRUX_EINVAL, "autotune needs a rank set, genotypes and 0 < P_c < 1");
  KRUX_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = std::min<int64_t>(S, 65536);
  const int64_t cap = 1 << 20;
  DevBuf out;
  KRUX_CUDA(ctx, out.ensure((size_t)cap * (sizeof(krux_hit) + 16)));
  krux_hit *hits = out.as<krux_hit>();
  double *H = reinterpret_cast<double *>(out.as<char>() + (size_t)cap * sizeof(krux_hit));
  double *P = H + cap;
  krux_opts o{};
  o.pthresh = pthresh;
  o.hit_capacity = cap;
  o.snp_end = n;
  struct Cand { int layout, nc, nA, ka; };
  std::vector<Cand> cands = {{-1, 0, 0, 0}};
  for (int layout : {1, 0})
    for (int nc : {4, 3, 2, 1})
      for (int nA : {2, 3, 4})
        for (int ka : {0, 64}) cands.push_back(Cand{layout, nc, nA, ka});
  const int s_layout = ctx->tune_layout, s_nc = ctx->tune_nc, s_nA = ctx->tune_nA,
            s_ka = ctx->tune_ka;
  const bool s_prof = ctx->profiling;
  const auto saved_tuned = ctx->tuned;
  ctx->tuned.erase(rs->Np);
  ctx->profiling = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 0.f;
  Cand best{-1, 0, 0, 0};
  bool any = false;
  krux_status result = KRUX_OK;
  for (const Cand &c : cands) {
    ctx->tune_layout = c.layout;
    ctx->tune_nc = c.nc;
    ctx->tune_nA = c.nA;
    ctx->tune_ka = c.ka;
    float ms = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      int64_t nh = 0;
      cudaEventRecord(e0, s);
      const krux_status st = krux_scan(ctx, rs, geno, S, ldg, &o, hits, H, P, &nh, stream);
      cudaEventRecord(e1, s);
      if (st == KRUX_ECUDA || st == KRUX_ETIMEOUT) {
        result = st;  // a real failure: stop tuning
        ok = false;
        break;
      }
      if (st != KRUX_OK && st != KRUX_EOVERFLOW) {
        ok = false;  // this shape does not fit
        break;
      }
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep == 1 || (rep == 2 && t < ms)) ms = t;  // best of the two timed runs
    }
    if (result != KRUX_OK) break;
    if (ok && (!any || ms < best_ms)) {
      any = true;
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tune_layout = s_layout;
  ctx->tune_nc = s_nc;
  ctx->tune_nA = s_nA;
  ctx->tune_ka = s_ka;
  ctx->profiling = s_prof;
  out.release();
  if (result != KRUX_OK) {
    ctx->tuned = saved_tuned;
    return result;
  }
  if (!any) {
    ctx->tuned = saved_tuned;
    return fail(ctx, KRUX_EUNSUPPORTED, "no launch shape ran");
  }
  ctx->tuned[rs->Np] = {best.layout, best.nc, best.nA, best.ka};
  if (shape_out) {
    shape_out[0] = best.layout;
    shape_out[1] = best.nc;
    shape_out[2] = best.nA;
    shape_out[3] = best.ka;
  }
  return KRUX_OK;
}

// Test hook: the launch plan for one group of N samples (no GPU needed).
extern "C" krux_status krux_debug_plan(int N, int with_nan, int layout, int nc, int nA, int ka,
                                       int32_t *out) {
  if (N < 1 || N > kMaxN || !out) return KRUX_EINVAL;
  krux_ctx tmp;
  tmp.tune_layout = layout;
  tmp.tune_nc = nc;
  tmp.tune_nA = nA;
  tmp.tune_ka = ka;
  const int lay = layout >= 0 ? layout : 1;
  const int atom = layout_atom(lay);
  const int Np = round_up(N, 16);
  const int kpad = round_up(Np, atom);
  // with_nan: 0 complete data, 1 the general form's 2-bit codes, 2 the plain form
  // (complete data, room for its hit-event ring), 3 the plain form's NaN variant
  // (its coefficient sets in place of the codes)
  if (with_nan < 0 || with_nan > 3) return KRUX_EINVAL;
  const bool plain = with_nan >= 2;
  if (plain && lay != 1) return KRUX_EUNSUPPORTED;
  const int codes_k = with_nan == 1 ? Np : (with_nan == 3 ? kCoefNanRows : 0);
  LaunchShape sh;
  if (!pick_launch_shape(&tmp, kpad, codes_k, sh, plain ? kEvRegion : 0)) return KRUX_EUNSUPPORTED;
  GroupDesc d;
  std::memset(&d, 0, sizeof d);
  d.Np = Np;
  d.n_atoms = (Np + atom - 1) / atom;
  d.codes = codes_k ? reinterpret_cast<const uint64_t *>(16) : nullptr;
  d.codes_k = codes_k;
  group_shape(sh, kpad, atom, d);
  // the plain forms: the whole K per rank stage, chunk pairs
  if (plain && (sh.ka != kpad || d.pair != 1 || d.nkb != 1)) return KRUX_EUNSUPPORTED;
  ScanParams p{};
  p.nc = d.nc;
  p.nA = sh.nA;
  p.kpad = std::max(codes_k, 16);
  p.ka = sh.ka;
  p.a_tile_bytes = 256 * sh.ka;
  p.b_region = sh.b_region;
  p.layout = lay;
  const size_t smem = scan_smem_bytes2(p.nc, p.nA, (size_t)p.a_tile_bytes, (size_t)p.b_region, p.kpad) +
                     (plain ? kEvRegion : 0);
  out[0] = sh.ka;
  out[1] = sh.nA;
  out[2] = sh.b_region;
  out[3] = d.nc;
  out[4] = d.nkb;
  out[5] = d.b_stride;
  out[6] = (int32_t)smem;
  const std::string why = validate_plan(p, std::vector<GroupDesc>{d}, smem);
  return why.empty() ? KRUX_OK : KRUX_EUNSUPPORTED;
}
