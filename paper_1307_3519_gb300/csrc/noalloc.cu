// noalloc.cu -- krux_scan_noalloc: the fused scan for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running under an allocator
// that owns the whole device (a framework's caching allocator, or a host that
// reserved the device memory up front), plugins loaded into such processes, and
// real-time paths where an allocation could block or fail.  This entry point
// runs the same kernels as krux_scan (rank transform, genotype packing, fused
// scan, FP64 finalisation) but takes every piece of scratch memory from one
// file-scope device array of fixed size.  The caller still passes its inputs
// and outputs.  Nothing here calls cudaMalloc, cudaFree or any allocating
// library routine.
//
// The array is a module global: every GPU that loads this library holds it
// until the process exits, and every call on a device shares it (the previous
// call's contents stay behind; what must start at zero is cleared by each call).
// Calls that overlap on the GPU therefore race; run them on one stream or
// serialise them.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace krux {
cudaError_t launch_pack2(const int8_t *geno, int64_t ldg, int N, int Np, const int64_t *snp_list,
                         int64_t snp_begin, int64_t n_snps, int64_t snp_out_base, double h1,
                         double h2, int allow_missing, int signed_df1, __half *B,
                         ChunkMeta *meta, uint64_t *codes, unsigned int *status, cudaStream_t s);
}  // namespace krux

using namespace krux;

namespace {

// ---- limits and the scratch layout (all sizes in bytes) --------------------
constexpr int kNaMaxT = 4096;        // traits
constexpr int kNaMaxN = 256;         // samples
constexpr int kNaSlice = 4096;       // SNPs packed and scanned per launch (any S is sliced)
constexpr int64_t kNaMaxHits = 262144;  // hit records stored per call (the count stays exact)
constexpr int kNaMaxItems = 1024;
constexpr int kNaRows = kNaMaxT;     // kNaMaxT is a multiple of the 128-trait tile
constexpr int kNaChunks = kNaSlice / kChunkSnps;

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffDesc = 0;                                               // GroupDesc
constexpr size_t kOffItems = al256(kOffDesc + sizeof(GroupDesc));            // WorkItem[]
constexpr size_t kOffCnt = al256(kOffItems + sizeof(WorkItem) * kNaMaxItems);  // counter, status
constexpr size_t kOffCfp = al256(kOffCnt + 64);                              // const double *[1]
constexpr size_t kOffA = al256(kOffCfp + 64);
constexpr size_t kOffLo = al256(kOffA + (size_t)kNaRows * kNaMaxN * 2);
constexpr size_t kOffEq = al256(kOffLo + (size_t)kNaMaxT * kNaMaxN * 2);
constexpr size_t kOffTie = al256(kOffEq + (size_t)kNaMaxT * kNaMaxN * 2);
constexpr size_t kOffK = al256(kOffTie + (size_t)kNaMaxT * 8);
constexpr size_t kOffTau = al256(kOffK + (size_t)kNaMaxT * 4);
constexpr size_t kOffCfac = al256(kOffTau + (size_t)kNaMaxT * 4);
constexpr size_t kOffNanCnt = al256(kOffCfac + (size_t)kNaMaxT * 8);
constexpr size_t kOffNanIdx = al256(kOffNanCnt + (size_t)kNaMaxT * 2);
constexpr size_t kOffTileNan = al256(kOffNanIdx + (size_t)kNaMaxT * kNaMaxN * 2);
constexpr size_t kOffB = al256(kOffTileNan + (size_t)(kNaRows / kTileM) * 4);
constexpr size_t kOffMeta = al256(kOffB + (size_t)kNaChunks * kChunkRows * kNaMaxN * 2);
constexpr size_t kOffCodes = al256(kOffMeta + (size_t)kNaChunks * sizeof(ChunkMeta));
constexpr size_t kOffAux = al256(kOffCodes + (size_t)kNaChunks * kNaMaxN * 16);
constexpr size_t kNaBytes = al256(kOffAux + (size_t)kNaMaxHits * sizeof(HitAux));
static_assert(kNaBytes <= (size_t)16 << 20, "no-alloc scratch must stay within 16 MiB");

// The scratch itself.  In host code `g_noalloc_scratch` only names the symbol:
// its device address comes from cudaGetSymbolAddress (set-up below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// ---- per-device set-up ------------------------------------------------------
constexpr int kNaMaxDevices = 64;
struct DeviceSetup {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};
DeviceSetup g_setup[kNaMaxDevices];
std::mutex g_setup_mu;

krux_status setup_device(int dev, DeviceSetup **out) {
  if (dev < 0 || dev >= kNaMaxDevices) return KRUX_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup &d = g_setup[dev];
  if (!d.ready) {
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return KRUX_ECUDA;
    if (!(major == 10 && minor == 3)) return KRUX_EUNSUPPORTED;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return KRUX_ECUDA;
    d.scratch = static_cast<unsigned char *>(p);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        fn == nullptr)
      return KRUX_ECUDA;
    d.encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    d.ready = true;
  }
  *out = &d;
  return KRUX_OK;
}

double na_h1(double p) {
  double lo = 0.0, hi = 40.0;
  for (int i = 0; i < 200; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (std::erfc(mid) > p) lo = mid; else hi = mid;
  }
  const double x = 0.5 * (lo + hi);
  return 2.0 * x * x;
}

bool na_encode(const DeviceSetup &d, CUtensorMap *map, const void *base, int Np, int64_t rows) {
  cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Np * 2};
  cuuint32_t box[2] = {16u, (cuuint32_t)kTileM};
  cuuint32_t estr[2] = {1, 1};
  return d.encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

#define NA_CUDA(call)                                   \
  do {                                                  \
    if ((call) != cudaSuccess) return KRUX_ECUDA;       \
  } while (0)

extern "C" krux_status krux_scan_noalloc(const float *expr, int T, int N, int64_t ld,
                                         const int8_t *geno, int64_t S, int64_t ldg,
                                         double pthresh, krux_hit *hits, double *hit_H,
                                         double *hit_p, int64_t hit_capacity, int64_t *n_hits,
                                         void *stream) {
  if (!n_hits) return KRUX_EINVAL;
  *n_hits = 0;
  if (!expr || T < 1 || T > kNaMaxT || N < 1 || N > kNaMaxN || ld < N || S < 0 ||
      (S > 0 && (!geno || ldg < N)) || S >= ((int64_t)1 << 31) || !(pthresh > 0.0 && pthresh < 1.0) ||
      hit_capacity < 0 || (hit_capacity > 0 && (!hits || !hit_H || !hit_p)) ||
      ((uintptr_t)hits & 15u) != 0)
    return KRUX_EINVAL;
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  DeviceSetup *d = nullptr;
  krux_status st = setup_device(dev, &d);
  if (st != KRUX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *sc = d->scratch;

  const int Np = (N + 15) / 16 * 16;
  const int rows_pad = (T + kTileM - 1) / kTileM * kTileM;
  const int n_ttiles = rows_pad / kTileM;
  RankDev r{};
  r.A = reinterpret_cast<__half *>(sc + kOffA);
  r.lo = reinterpret_cast<uint16_t *>(sc + kOffLo);
  r.eq = reinterpret_cast<uint16_t *>(sc + kOffEq);
  r.tie = reinterpret_cast<int64_t *>(sc + kOffTie);
  r.K = reinterpret_cast<int32_t *>(sc + kOffK);
  r.tau = reinterpret_cast<float *>(sc + kOffTau);
  r.cfac = reinterpret_cast<double *>(sc + kOffCfac);
  r.nan_cnt = reinterpret_cast<uint16_t *>(sc + kOffNanCnt);
  r.nan_idx = reinterpret_cast<uint16_t *>(sc + kOffNanIdx);
  r.tile_nan = reinterpret_cast<uint32_t *>(sc + kOffTileNan);
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(sc + kOffCnt);
  unsigned int *status = reinterpret_cast<unsigned int *>(sc + kOffCnt + 16);
  const double **cfacptr = reinterpret_cast<const double **>(sc + kOffCfp);
  __half *B = reinterpret_cast<__half *>(sc + kOffB);
  ChunkMeta *meta = reinterpret_cast<ChunkMeta *>(sc + kOffMeta);
  uint64_t *codes = reinterpret_cast<uint64_t *>(sc + kOffCodes);
  HitAux *aux = reinterpret_cast<HitAux *>(sc + kOffAux);
  GroupDesc *gdesc = reinterpret_cast<GroupDesc *>(sc + kOffDesc);
  WorkItem *ditems = reinterpret_cast<WorkItem *>(sc + kOffItems);
  const int64_t cap = std::min<int64_t>(hit_capacity, kNaMaxHits);

  // the previous call's data stays in the array: clear what must start at zero
  NA_CUDA(cudaMemsetAsync(sc + kOffCnt, 0, 64, s));
  NA_CUDA(cudaMemsetAsync(r.A, 0, (size_t)rows_pad * Np * 2, s));
  NA_CUDA(cudaMemsetAsync(r.tile_nan, 0, (size_t)n_ttiles * 4, s));
  const double *cf = r.cfac;
  NA_CUDA(cudaMemcpyAsync(cfacptr, &cf, sizeof cf, cudaMemcpyHostToDevice, s));
  NA_CUDA(launch_rank(expr, T, N, ld, Np, rows_pad, r, s));

  const double h1 = na_h1(pthresh), h2 = -2.0 * std::log(pthresh);
  // shape for this Np with the 32-byte-swizzle layout (largest resident chunk count)
  int nc = 0, nA = 0;
  for (int c = 4; c >= 1 && nc == 0; --c)
    for (int a = 4; a >= 2; --a)
      if (scan_smem_bytes(c, a, Np) <= 232448) {
        nc = c;
        nA = a;
        break;
      }
  if (nc == 0) return KRUX_EUNSUPPORTED;

  for (int64_t b = 0; b < S; b += kNaSlice) {
    const int64_t n = std::min<int64_t>(kNaSlice, S - b);
    const int64_t nch = (n + kChunkSnps - 1) / kChunkSnps;
    NA_CUDA(launch_pack2(geno, ldg, N, Np, nullptr, b, n, 0, h1, h2, 0, 0, B, meta, codes, status, s));
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    if (!na_encode(*d, &g.tmA, r.A, Np, rows_pad) || !na_encode(*d, &g.tmB, B, Np, nch * kChunkRows))
      return KRUX_ECUDA;
    g.meta = meta;
    g.codes = codes;
    g.codes_k = Np;
    g.tau = r.tau;
    g.cfac = r.cfac;
    g.nan_cnt = r.nan_cnt;
    g.nan_idx = r.nan_idx;
    g.tile_nan = r.tile_nan;
    g.hits = hits;
    g.aux = aux;
    g.counter = counter;
    g.capacity = cap;
    g.T = T;
    g.N = N;
    g.Np = Np;
    g.n_ttiles = n_ttiles;
    g.rows_per_agroup = rows_pad;
    g.n_agroups = 1;
    g.nchunks = (int32_t)nch;
    g.n_atoms = Np / 16;
    g.group_id = 0;
    g.nc = nc;
    g.b_stride = 256 * Np;
    g.nkb = 1;
    // work items: one B tile of nc chunks against all trait tiles, split to fill the SMs
    WorkItem items[kNaMaxItems];
    const int64_t nbt = (nch + nc - 1) / nc;
    int split = 1;
    while (split < n_ttiles && nbt * (split + 1) <= d->sm_count && nbt * (split + 1) <= kNaMaxItems) ++split;
    int ni = 0;
    for (int64_t bt = 0; bt < nbt; ++bt)
      for (int k = 0; k < split; ++k) {
        const int s0 = (int)((int64_t)n_ttiles * k / split), s1 = (int)((int64_t)n_ttiles * (k + 1) / split);
        if (s1 > s0) items[ni++] = WorkItem{0, (int32_t)bt, s0, s1};
      }
    NA_CUDA(cudaMemcpyAsync(gdesc, &g, sizeof g, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(ditems, items, sizeof(WorkItem) * ni, cudaMemcpyHostToDevice, s));
    ScanParams p{};
    p.groups = gdesc;
    p.items = ditems;
    p.n_items = ni;
    p.nc = nc;
    p.nA = nA;
    p.kpad = Np;
    p.ka = Np;
    p.a_tile_bytes = 256 * Np;
    p.b_region = nc * 256 * Np;
    p.layout = 1;
    p.margin = 1e-4f;
    p.dense = 0;
    p.pthresh = pthresh;
    p.h1 = (float)h1;
    p.h2 = (float)h2;
    p.status = status;
    p.timeout_cycles = 4000000000LL;
    p.signed_coef = 0;
    p.seg_cap = 0;  // hits go straight to the caller's list
    // the rank set may hold NaN: the kernel form with exact per-pair group sizes for
    // traits with NaN (traits without NaN take the ordinary hot test there)
    p.has_nan = 1;
    const int grid = std::min(ni, d->sm_count);
    NA_CUDA(launch_scan(p, grid, scan_smem_bytes(nc, nA, Np), s));
  }
  unsigned long long cnt = 0;
  unsigned int hst[2] = {0, 0};
  NA_CUDA(cudaMemcpyAsync(&cnt, counter, 8, cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaMemcpyAsync(hst, status, 8, cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  if (hst[0] & kDevBadCode) return KRUX_EINVAL;        // genotype code outside {-1,0,1,2}
  if (hst[0] & kDevMissing) return KRUX_EUNSUPPORTED;  // a -1 code (packed as complete data)
  if (hst[0] & kDevTimeout) return KRUX_ETIMEOUT;
  const int64_t stored = std::min<int64_t>((int64_t)cnt, cap);
  if (stored > 0) {
    NA_CUDA(launch_finalize(hits, aux, stored, cfacptr, hit_H, hit_p, s, nullptr, 0, 0.0, 1.0, pthresh));
    NA_CUDA(cudaStreamSynchronize(s));
  }
  *n_hits = (int64_t)cnt;
  return (int64_t)cnt > cap ? KRUX_EOVERFLOW : KRUX_OK;
}
