// ------------------------------------------------------------------------
// Learned surrogate (surrogate.cuh): a per-agent message-passing network
// that predicts a whole world step of the 16-agent walled sphere world, with
// the plain step as the fallback for envs whose prediction overlaps.

#include "gemm_tc.cuh"
#include "host.h"
#include "surrogate_fused.cuh"

using namespace vmas_host;

namespace {

using vmas::sur::bf16;
namespace sur = vmas::sur;

using namespace vmas::sur;  // parameter offsets kOff*
constexpr int kSurParams = vmas::sur::kParams;
constexpr int kSplitCap = 256;  // split-K / column-sum partial blocks
constexpr int kWgradMinK = 4096;  // K from which weight gradients take wgrad_tc_kernel

// K-major (transposed) bfloat16 copies of the weights whose products with an
// upstream gradient are plain row-major GEMMs in the backward, so that they
// too run on the tensor-core GEMM: W2^T [128][128], W1^T [80][128],
// We2^T [64][64].
constexpr int kOffW2T = 0, kOffW1T = 128 * 128, kOffWe2T = kOffW1T + 80 * 128,
              kOffW3T = kOffWe2T + 64 * 64, kTransposed = kOffW3T + 128 * 8;

// 0: the tcgen05 GEMM wherever the shape allows it (the default);
// 1: the warp-mma GEMM only (for A/B comparisons).  Process-wide.
int g_gemm_engine = 0;
std::atomic<long long> g_tc_launches{0};  // tcgen05 GEMM launches so far
std::atomic<int> g_tc_timeout_test{0};    // vmas_debug_gemm_timeout

}  // namespace

struct vmas_surrogate {
  int device = 0;
  int cap = 0;  // envs
  int mode = VMAS_SUR_FUSED;
  int n_sm = 0;
  bool fused_ready = false;  // shared-memory opt-in of the fused kernel done
  int adam_t = 0;
  float *p32 = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  bf16 *pbf = nullptr;
  bf16 *pbfT = nullptr;  // transposed weight copies (kOff*T)
  int *err = nullptr;    // device error word of the surrogate's kernels
  // forward
  bf16 *node = nullptr, *edge = nullptr, *he = nullptr, *zin = nullptr, *h1 = nullptr,
       *h2 = nullptr;
  float *mask = nullptr, *ze2 = nullptr, *out = nullptr;
  // training (allocated on first use)
  float *ze1 = nullptr, *z1 = nullptr, *z2 = nullptr;
  float *d_out = nullptr, *g128 = nullptr, *d_zin = nullptr, *ge = nullptr;
  bf16 *d_outbf = nullptr, *g128bf = nullptr, *gebf = nullptr;
  float *part = nullptr, *loss_part = nullptr, *save = nullptr, *target = nullptr;
  int *list = nullptr, *list_len = nullptr;
  // compact edges: the used neighbour slots, in slot-major order
  bf16 *edgec = nullptr;                         // [RK][16] features of the used slots
  int *epos = nullptr, *emap = nullptr;          // [RK] slot -> position (-1), position -> slot
  int *escan = nullptr, *etotal = nullptr;       // block sums; the count
  int *h_total = nullptr;                        // pinned host copy of the count
  int n_edges = 0;                               // used slots of the last forward
};

namespace {

void free_sur(vmas_surrogate *s) {
  if (!s) return;
  void *ptrs[] = {s->p32,   s->grad,  s->adam_m, s->adam_v, s->pbf,    s->node,   s->edge,
                  s->he,    s->zin,   s->h1,     s->h2,     s->mask,   s->ze2,    s->out,
                  s->ze1,   s->z1,    s->z2,     s->d_out,  s->g128,   s->d_zin,  s->ge,
                  s->d_outbf, s->g128bf, s->gebf, s->part,  s->loss_part, s->save, s->target,
                  s->list,  s->list_len, s->pbfT, s->err, s->edgec, s->epos, s->emap,
                  s->escan, s->etotal};
  for (void *q : ptrs) cudaFree(q);
  if (s->h_total) cudaFreeHost(s->h_total);
  delete s;
}

template <typename T>
bool dalloc(T **ptr, size_t count) {
  return cudaMalloc((void **)ptr, (count > 0 ? count : 1) * sizeof(T)) == cudaSuccess;
}

// Network rows per env of a world (16 agents, or 16 agents + 4 boxes) and
// the width of its training targets (x y vx vy, plus theta omega for boxes).
int nodes_of(const vmas_world *w) { return w->sur_layout == 2 ? sur::kNodesMax : sur::kAgents; }
int target_width(const vmas_world *w) { return w->sur_layout == 2 ? 6 : 4; }

int ensure_training(vmas_surrogate *s) {
  if (s->ze1) return VMAS_OK;
  const size_t R = (size_t)s->cap * sur::kNodesMax, RK = R * sur::kK;
  const bool ok = dalloc(&s->ze1, RK * 64) && dalloc(&s->z1, R * 128) && dalloc(&s->z2, R * 128) &&
                  dalloc(&s->d_out, R * 8) && dalloc(&s->d_outbf, R * 8) &&
                  dalloc(&s->g128, R * 128) && dalloc(&s->g128bf, R * 128) &&
                  dalloc(&s->d_zin, R * 80) && dalloc(&s->ge, RK * 64) &&
                  dalloc(&s->gebf, RK * 64) && dalloc(&s->save, R * 6) &&
                  dalloc(&s->target, R * 6);
  if (!ok) {
    cudaGetLastError();
    return fail(VMAS_ENOMEM, "cudaMalloc failed for the surrogate's training buffers");
  }
  return VMAS_OK;
}

unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// cuTensorMapEncodeTiled, reached through the runtime (no link to the
// driver library); null when unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  }
  return fn;
}

// Tensor map of a row-major bfloat16 matrix [rows][K] (leading dimension ld
// elements): boxes of 64 K-elements (128 bytes, the swizzle span) by
// box_rows rows, 128-byte swizzle, zero fill past the edges.
bool tc_map(CUtensorMap *m, const bf16 *p, int rows, int K, int ld, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(p), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C = A B^T-stored (B[n][k]) on the tensor cores; false (nothing enqueued)
// when the shape or a tensor map does not allow it.
bool gemm_tc(cudaStream_t st, int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb,
             const float *bias, int act, float *out_f32, int ldc_f, bf16 *out_bf, int ldc_b,
             int *err, int *rc) {
  auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  if (g_gemm_engine != 0 || !err || M < 1 || N < 1 || N > 128 || K < 8 || K > 128 || K % 8 ||
      lda % 8 || ldb % 8 || !al16(A) || !al16(B))
    return false;
  sur::TcGemmArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.n_pad = (N + 15) / 16 * 16;
  g.katoms = (K + 63) / 64;
  g.bias = bias; g.act = act;
  g.out_f32 = out_f32; g.ldc_f = ldc_f; g.out_bf = out_bf; g.ldc_b = ldc_b;
  g.err = err;
  g.vec_f = out_f32 && al16(out_f32) && ldc_f % 4 == 0;
  g.vec_b = out_bf && al16(out_bf) && ldc_b % 8 == 0;
  g.extra_tx = g_tc_timeout_test.load() ? 16u : 0u;
  CUtensorMap ma, mb;
  if (!tc_map(&ma, A, M, K, lda, sur::kTcM) || !tc_map(&mb, B, N, K, ldb, g.n_pad)) return false;
  // outputs through TMA stores: boxes of 32 rows x 32 bytes, no swizzle
  CUtensorMap mc{}, mcb{};
  {
    EncodeTiledFn fn = encode_tiled();
    auto out_map = [&](CUtensorMap *m, void *p, CUtensorMapDataType t, int esize, int ld) {
      if (!fn || !al16(p) || ((size_t)ld * esize) % 16) return false;
      const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
      const cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
      const cuuint32_t box[2] = {(cuuint32_t)(32 / esize), 32u};
      const cuuint32_t estr[2] = {1u, 1u};
      return fn(m, t, 2, p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    g.tma_st = (out_f32 || out_bf) &&
               (!out_f32 || out_map(&mc, out_f32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ldc_f)) &&
               (!out_bf || out_map(&mcb, out_bf, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ldc_b));
  }
  // SM count and the shared-memory opt-in, once per process (thread-safe
  // initialisation); 0 when the set-up failed (the warp-mma GEMM then runs)
  static const int n_sm = []() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(sur::gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sur::tc_smem_bytes(2, 128)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return sms;
  }();
  if (!n_sm) return false;
  const int tiles = (M + sur::kTcM - 1) / sur::kTcM;
  const int grid = std::min(tiles, 2 * n_sm);
  sur::gemm_tc_kernel<<<grid, sur::kTcThreads, sur::tc_smem_bytes(g.katoms, g.n_pad), st>>>(ma, mb, mc,
                                                                                          mcb, g);
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++g_tc_launches;
  *rc = e == cudaSuccess ? VMAS_OK : cuda_fail(e, "gemm_tc_kernel launch");
  return true;
}

// Weight gradient C [M][N] = A^T B with A [K][M], B [K][N] (row-major,
// leading dimensions lda, ldb) on the tensor cores (wgrad_tc_kernel, split
// K over at most `cap` CTAs, partials in `part` [cap][M][N], reduced into
// out [M][N]); false (nothing enqueued) when the shape, the buffers or a
// tensor map do not allow it.
bool gemm_tc_wgrad(cudaStream_t st, int M, int N, int K, const bf16 *A, int lda, const bf16 *B,
                   int ldb, float *out, float *part, int cap, int *err, int *rc) {
  auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  if (g_gemm_engine != 0 || !err || !part || cap < 1 || M < 1 || N < 1 || M > 128 || N > 128 ||
      K < kWgradMinK || lda < M || ldb < N || lda % 8 || ldb % 8 || !al16(A) || !al16(B))
    return false;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  // MN-major tiles: 64 columns (128 bytes, the swizzle span) by 64 rows
  auto map = [&](CUtensorMap *m, const bf16 *p, int width, int ld) {
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)K};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {64u, 64u};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(p), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  CUtensorMap ma, mb;
  if (!map(&ma, A, M, lda) || !map(&mb, B, N, ldb)) return false;
  static const bool smem_ok = []() {
    const bool ok = cudaFuncSetAttribute(sur::wgrad_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sur::wgrad_smem_bytes()) == cudaSuccess;
    cudaGetLastError();
    return ok;
  }();
  if (!smem_ok) return false;
  sur::WgradArgs g{};
  g.M = M;
  g.N = N;
  g.n_mma = N > 64 ? 128 : 64;
  g.nblocks = (K + 63) / 64;
  g.kb = (g.nblocks + cap - 1) / cap;              // blocks per CTA
  const int grid = (g.nblocks + g.kb - 1) / g.kb;  // <= cap, every CTA has a block
  g.part = part;
  g.err = err;
  g.vec = N % 4 == 0;
  g.extra_tx = g_tc_timeout_test.load() ? 16u : 0u;
  sur::wgrad_tc_kernel<<<grid, 128, sur::wgrad_smem_bytes(), st>>>(ma, mb, g);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    ++g_tc_launches;
    const size_t MN = (size_t)M * N;
    sur::sum_partials_kernel<<<blocks_for(MN, 256), 256, 0, st>>>(out, part, grid, MN);
    e = cudaGetLastError();
  }
  *rc = e == cudaSuccess ? VMAS_OK : cuda_fail(e, "wgrad_tc_kernel launch");
  return true;
}

// C = A B (+ bias, GELU): on the tensor cores (gemm_tc_kernel) when A is
// row-major, B stored [N][K], K a multiple of 8 up to 128, N up to 128 and
// an error word is given; otherwise through gemm_bf16_kernel (warp mma), where
// `splits` > 1 sums K in chunks into part, reduced into out_f32 (then no
// bias / bf16 output).
int gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, const bf16 *A, int lda,
         const bf16 *B, int ldb, const float *bias, int act, float *out_f32, int ldc_f,
         bf16 *out_bf, int ldc_b, float *part = nullptr, int splits = 1, int *err = nullptr) {
  if (M == 0 || N == 0) return VMAS_OK;
  if (!ta && tb && splits == 1) {
    int rc = VMAS_OK;
    if (gemm_tc(st, M, N, K, A, lda, B, ldb, bias, act, out_f32, ldc_f, out_bf, ldc_b, err, &rc))
      return rc;
  }
  if (ta && !tb && splits > 1 && !bias && !act && !out_bf && out_f32 && ldc_f == N) {
    int rc = VMAS_OK;
    if (gemm_tc_wgrad(st, M, N, K, A, lda, B, ldb, out_f32, part, splits, err, &rc)) return rc;
  }
  sur::GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
  g.bias = bias; g.act = act;
  g.ldc_f = ldc_f; g.out_bf = out_bf; g.ldc_b = ldc_b;
  if (splits > 1 && K > 0) {
    int chunk = (K + splits - 1) / splits;
    chunk = (chunk + sur::kBK - 1) / sur::kBK * sur::kBK;
    splits = (K + chunk - 1) / chunk;
    g.kchunk = chunk;
    g.out_f32 = part;
    g.ldc_f = N;
  } else {
    splits = 1;
    g.kchunk = K > 0 ? K : 1;
    g.out_f32 = out_f32;
  }
  const dim3 grid(blocks_for((size_t)M, sur::kBM), blocks_for((size_t)N, sur::kBN), splits);
  if (!ta && !tb) sur::gemm_bf16_kernel<false, false><<<grid, 128, 0, st>>>(g);
  else if (!ta && tb) sur::gemm_bf16_kernel<false, true><<<grid, 128, 0, st>>>(g);
  else if (ta && !tb) sur::gemm_bf16_kernel<true, false><<<grid, 128, 0, st>>>(g);
  else sur::gemm_bf16_kernel<true, true><<<grid, 128, 0, st>>>(g);
  VMAS_CUDA(cudaGetLastError());
  if (g.out_f32 == part && part) {
    const size_t MN = (size_t)M * N;
    sur::sum_partials_kernel<<<blocks_for(MN, 256), 256, 0, st>>>(out_f32, part, splits, MN);
    VMAS_CUDA(cudaGetLastError());
  }
  return VMAS_OK;
}

// Column sums of x [M][N] (N <= 128) into out [N]: up to 4,096 row chunks
// summed in parallel, then the chunk sums per column (two stages).
// Row chunks of the first column-sum stage for M rows.
void col_chunks(int M, int *chunks, int *chunk) {
  *chunks = std::max(1, std::min(4096, (M + 255) / 256));
  *chunk = std::max(1, (M + *chunks - 1) / *chunks);
}

// Stages 2 and 3 of a column sum: the `chunks` partial rows in part [chunks][N]
// into 64 groups, then the groups into out [N].
int col_sum_finish(cudaStream_t st, float *out, float *part, int chunks, int N) {
  const int groups = std::min(64, chunks), per = (chunks + groups - 1) / groups;
  float *part2 = part + (size_t)chunks * N;
  sur::col_sum_kernel<<<groups, 128, 0, st>>>(part2, part, chunks, N, per);
  VMAS_CUDA(cudaGetLastError());
  sur::sum_partials_kernel<<<1, 128, 0, st>>>(out, part2, groups, (size_t)N);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

// d_zbf = bf(d_h gelu'(z)) over [M][N] (N <= 128) and the bias gradient
// out [N] = the column sums of the FP32 d_h gelu'(z), in col_sum's order.
int gelu_back_sum(cudaStream_t st, float *out, const float *d_h, const float *z, bf16 *d_zbf,
                  int M, int N, float *part) {
  int chunks, chunk;
  col_chunks(M, &chunks, &chunk);
  sur::gelu_back_sum_kernel<<<chunks, N <= 64 ? 64 : 128, 0, st>>>(M, N, d_h, z, d_zbf, part, chunk);
  VMAS_CUDA(cudaGetLastError());
  return col_sum_finish(st, out, part, chunks, N);
}

int col_sum(cudaStream_t st, float *out, const float *x, int M, int N, float *part) {
  int chunks, chunk;
  col_chunks(M, &chunks, &chunk);
  sur::col_sum_kernel<<<chunks, 128, 0, st>>>(part, x, M, N, chunk);
  VMAS_CUDA(cudaGetLastError());
  return col_sum_finish(st, out, part, chunks, N);
}

int sur_check(vmas_surrogate *s, vmas_world *w, const float *d_actions) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  if (!w) return fail(VMAS_EINVAL, "world is NULL");
  if (!w->sur_ok)
    return fail(VMAS_EINVAL,
                "world layout is not 16 actuated agent spheres, optionally 4 actuated boxes, "
                "then 4 fixed lines");
  if (w->E > s->cap)
    return fail(VMAS_EINVAL, "world has " + std::to_string(w->E) + " envs, surrogate capacity " +
                                 std::to_string(s->cap));
  if (w->E > 0 && !d_actions) return fail(VMAS_EINVAL, "d_actions is NULL");
  return VMAS_OK;
}

// Features of the world's current state, then the network; train = true also
// keeps the FP32 pre-activations the backward needs.
int sur_forward(vmas_surrogate *s, vmas_world *w, const float *d_actions, bool train,
                cudaStream_t st) {
  const int E = w->E;
  const int R = E * nodes_of(w), RK = R * sur::kK;
  if (E == 0) return VMAS_OK;
  sur::FeatureArgs f{};
  const size_t EN = (size_t)E * w->N;
  f.E = E; f.N = w->N; f.A = w->A; f.nodes = nodes_of(w);
  f.px = w->planes; f.py = w->planes + EN; f.vx = w->planes + 2 * EN; f.vy = w->planes + 3 * EN;
  f.th = w->planes + 4 * EN; f.om = w->planes + 5 * EN;
  f.param = w->param; f.kind = w->kind; f.actions = d_actions;
  f.node = s->node; f.edge = s->edge; f.mask = s->mask;
  sur::features_kernel<<<blocks_for(R, 128), 128, 0, st>>>(f);
  VMAS_CUDA(cudaGetLastError());
  const bf16 *W = s->pbf;
  const float *P = s->p32;
  int rc;
  // the used neighbour slots, compacted; their count comes back to the host
  // (one stream synchronisation) to size the edge GEMMs
  const int nb = (int)blocks_for((size_t)RK, sur::kScanBlock);
  sur::edge_scan_blocks_kernel<<<nb, sur::kScanThreads, 0, st>>>((size_t)RK, s->mask, s->epos,
                                                                 s->escan);
  sur::edge_scan_sums_kernel<<<1, 1024, 0, st>>>(nb, s->escan, s->etotal);
  sur::edge_compact_kernel<<<blocks_for((size_t)RK, 256), 256, 0, st>>>(
      (size_t)RK, s->epos, s->escan, s->edge, s->edgec, s->emap);
  VMAS_CUDA(cudaGetLastError());
  VMAS_CUDA(cudaMemcpyAsync(s->h_total, s->etotal, sizeof(int), cudaMemcpyDeviceToHost, st));
  VMAS_CUDA(cudaStreamSynchronize(st));
  const int RE = *s->h_total;
  if (RE < 0 || RE > RK) return fail(VMAS_EDEVICE, "edge count out of range");
  s->n_edges = RE;
  // edge MLP on the used slots
  if (RE > 0) {
    if ((rc = gemm(st, false, true, RE, 64, 16, s->edgec, 16, W + kOffWe1, 16, P + kOffbe1, 1,
                   train ? s->ze1 : nullptr, 64, s->he, 64, nullptr, 1, s->err)))
      return rc;
    if ((rc = gemm(st, false, true, RE, 64, 64, s->he, 64, W + kOffWe2, 64, P + kOffbe2, 0, s->ze2,
                   64, nullptr, 0, nullptr, 1, s->err)))
      return rc;
  }
  sur::aggregate_compact_kernel<<<blocks_for((size_t)R * 4, 256), 256, 0, st>>>(
      R, s->ze2, s->mask, s->epos, s->node, s->zin);
  VMAS_CUDA(cudaGetLastError());
  // node MLP
  if ((rc = gemm(st, false, true, R, 128, 80, s->zin, 80, W + kOffW1, 80, P + kOffb1, 1,
                 train ? s->z1 : nullptr, 128, s->h1, 128, nullptr, 1, s->err)))
    return rc;
  if ((rc = gemm(st, false, true, R, 128, 128, s->h1, 128, W + kOffW2, 128, P + kOffb2, 1,
                 train ? s->z2 : nullptr, 128, s->h2, 128, nullptr, 1, s->err)))
    return rc;
  return gemm(st, false, true, R, 8, 128, s->h2, 128, W + kOffW3, 128, P + kOffb3, 0, s->out, 8,
              nullptr, 0, nullptr, 1, s->err);
}

// Loss against target [R][tw] and the gradient into s->grad (after
// sur_forward with train = true), for E envs of `nodes` rows each.
int sur_backward(vmas_surrogate *s, int E, int nodes, int tw, const float *target, float *d_loss,
                 cudaStream_t st) {
  const int R = E * nodes;
  const float count = (float)E * (float)(sur::kAgents * 4 + (nodes - sur::kAgents) * 6);
  float *G = s->grad;
  VMAS_CUDA(cudaMemsetAsync(G, 0, kSurParams * sizeof(float), st));
  if (E == 0) {
    if (d_loss) VMAS_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
    return VMAS_OK;
  }
  const int lb = (int)blocks_for((size_t)R * 8, 256);
  sur::loss_kernel<<<lb, 256, 0, st>>>(R, nodes, tw, count, s->out, target, s->d_out, s->d_outbf,
                                       s->loss_part);
  VMAS_CUDA(cudaGetLastError());
  if (d_loss) {
    sur::finish_loss_kernel<<<1, 256, 0, st>>>(s->loss_part, lb, count, d_loss);
    VMAS_CUDA(cudaGetLastError());
  }
  int rc;
  const int sp = kSplitCap;
  // output layer
  if ((rc = gemm(st, true, false, 8, 128, R, s->d_outbf, 8, s->h2, 128, nullptr, 0, G + kOffW3,
                 128, nullptr, 0, s->part, sp, s->err)))
    return rc;
  if ((rc = col_sum(st, G + kOffb3, s->d_out, R, 8, s->part))) return rc;
  if ((rc = gemm(st, false, true, R, 128, 8, s->d_outbf, 8, s->pbfT + kOffW3T, 8, nullptr, 0,
                 s->g128, 128, nullptr, 0, nullptr, 1, s->err)))
    return rc;
  // node layer 2
  // (the bias gradient first: the weight gradient reuses the partial buffer)
  if ((rc = gelu_back_sum(st, G + kOffb2, s->g128, s->z2, s->g128bf, R, 128, s->part))) return rc;
  if ((rc = gemm(st, true, false, 128, 128, R, s->g128bf, 128, s->h1, 128, nullptr, 0, G + kOffW2,
                 128, nullptr, 0, s->part, sp, s->err)))
    return rc;
  if ((rc = gemm(st, false, true, R, 128, 128, s->g128bf, 128, s->pbfT + kOffW2T, 128, nullptr, 0,
                 s->g128, 128, nullptr, 0, nullptr, 1, s->err)))
    return rc;
  // node layer 1
  if ((rc = gelu_back_sum(st, G + kOffb1, s->g128, s->z1, s->g128bf, R, 128, s->part))) return rc;
  if ((rc = gemm(st, true, false, 128, 80, R, s->g128bf, 128, s->zin, 80, nullptr, 0, G + kOffW1, 80,
                 nullptr, 0, s->part, sp, s->err)))
    return rc;
  if ((rc = gemm(st, false, true, R, 80, 128, s->g128bf, 128, s->pbfT + kOffW1T, 128, nullptr, 0,
                 s->d_zin, 80, nullptr, 0, nullptr, 1, s->err)))
    return rc;
  // edge layer 2 (through the masked sum), on the used slots of the forward
  const int RE = s->n_edges;
  if (RE == 0) return VMAS_OK;  // no edge: the edge weights' gradients stay zero
  {  // the bias gradient first: the weight gradient reuses the partial buffer
    int chunks, chunk;
    col_chunks(RE, &chunks, &chunk);
    sur::edge_back_sum_kernel<<<chunks, 64, 0, st>>>(R, RE, s->d_zin, s->mask, s->emap, s->ze2,
                                                     s->gebf, s->part, chunk);
    VMAS_CUDA(cudaGetLastError());
    if ((rc = col_sum_finish(st, G + kOffbe2, s->part, chunks, 64))) return rc;
  }
  if ((rc = gemm(st, true, false, 64, 64, RE, s->gebf, 64, s->he, 64, nullptr, 0, G + kOffWe2, 64,
                 nullptr, 0, s->part, sp, s->err)))
    return rc;
  if ((rc = gemm(st, false, true, RE, 64, 64, s->gebf, 64, s->pbfT + kOffWe2T, 64, nullptr, 0, s->ge,
                 64, nullptr, 0, nullptr, 1, s->err)))
    return rc;
  // edge layer 1
  if ((rc = gelu_back_sum(st, G + kOffbe1, s->ge, s->ze1, s->gebf, RE, 64, s->part))) return rc;
  return gemm(st, true, false, 64, 16, RE, s->gebf, 64, s->edgec, 16, nullptr, 0, G + kOffWe1, 16,
              nullptr, 0, s->part, sp, s->err);
}

int refresh_transposed(vmas_surrogate *s, cudaStream_t st);

int sur_adam(vmas_surrogate *s, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  ++s->adam_t;
  const float c1 = (float)(1.0 - std::pow((double)b1, s->adam_t));
  const float c2 = (float)(1.0 - std::pow((double)b2, s->adam_t));
  sur::adam_kernel<<<blocks_for(kSurParams, 256), 256, 0, st>>>(
      kSurParams, s->p32, s->grad, s->adam_m, s->adam_v, s->pbf, lr, b1, b2, eps, c1, c2);
  VMAS_CUDA(cudaGetLastError());
  return refresh_transposed(s, st);
}

// The fused inference kernel over the world's envs: network output into
// out (may be NULL); apply = true also applies the prediction and lists the
// fallback envs.
int sur_fused(vmas_surrogate *s, vmas_world *w, const float *d_actions, float *out, bool apply,
              float limit, cudaStream_t st) {
  const int E = w->E;
  if (E == 0) return VMAS_OK;
  const size_t smem = sur::fused_smem_bytes();
  if (!s->fused_ready) {  // > 48 KB of dynamic shared memory needs an opt-in
    VMAS_CUDA(cudaFuncSetAttribute(sur::sur_fused_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    s->fused_ready = true;
  }
  sur::FusedArgs a{};
  const size_t EN = (size_t)E * w->N;
  a.E = E; a.N = w->N; a.A = w->A;
  a.px = w->planes; a.py = w->planes + EN; a.vx = w->planes + 2 * EN; a.vy = w->planes + 3 * EN;
  a.param = w->param; a.actions = d_actions;
  a.w = s->pbf; a.p = s->p32;
  a.out = out; a.apply = apply ? 1 : 0; a.limit = limit;
  a.list = s->list; a.list_len = s->list_len;
  const int need = (E + sur::kFusedWarpsPerCta - 1) / sur::kFusedWarpsPerCta;
  const int grid = std::max(1, std::min(need, s->n_sm));
  sur::sur_fused_kernel<<<grid, sur::kFusedWarpsPerCta * 32, smem, st>>>(a);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

__global__ void f32_to_bf16_kernel(const float *x, bf16 *y, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = __float2bfloat16_rn(x[t]);
}

// The transposed weight copies from the bfloat16 weights.
__global__ void transpose_weights_kernel(const bf16 *w, bf16 *wt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 128 * 128) {  // W2 [128][128]
    const int o = t / 128, i = t % 128;
    wt[kOffW2T + i * 128 + o] = w[kOffW2 + t];
  } else if (t < 128 * 128 + 128 * 80) {  // W1 [128][80]
    const int q = t - 128 * 128, o = q / 80, i = q % 80;
    wt[kOffW1T + i * 128 + o] = w[kOffW1 + q];
  } else if (t < kOffW3T) {  // We2 [64][64]
    const int q = t - 128 * 128 - 128 * 80, o = q / 64, i = q % 64;
    wt[kOffWe2T + i * 64 + o] = w[kOffWe2 + q];
  } else if (t < kTransposed) {  // W3 [8][128]
    const int q = t - kOffW3T, o = q / 128, i = q % 128;
    wt[kOffW3T + i * 8 + o] = w[kOffW3 + q];
  }
}

int refresh_transposed(vmas_surrogate *s, cudaStream_t st) {
  transpose_weights_kernel<<<blocks_for(kTransposed, 256), 256, 0, st>>>(s->pbf, s->pbfT);
  VMAS_CUDA(cudaGetLastError());
  return VMAS_OK;
}

}  // namespace

extern "C" {

int vmas_sur_param_count(void) { return kSurParams; }

int vmas_sur_create(int32_t max_envs, vmas_surrogate **out) {
  if (!out) return fail(VMAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_envs < 0 || max_envs > (1 << 22))
    return fail(VMAS_EINVAL, "max_envs must be 0.." + std::to_string(1 << 22));
  vmas_surrogate *s = new vmas_surrogate();
  cudaGetDevice(&s->device);
  if (cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      s->n_sm < 1) {
    cudaGetLastError();
    s->n_sm = 1;
  }
  s->cap = max_envs;
  const size_t R = (size_t)max_envs * sur::kNodesMax, RK = R * sur::kK;
  const bool ok =
      dalloc(&s->p32, kSurParams) && dalloc(&s->grad, kSurParams) && dalloc(&s->adam_m, kSurParams) &&
      dalloc(&s->adam_v, kSurParams) && dalloc(&s->pbf, kSurParams) && dalloc(&s->node, R * 16) &&
      dalloc(&s->edge, RK * 16) && dalloc(&s->he, RK * 64) && dalloc(&s->zin, R * 80) &&
      dalloc(&s->h1, R * 128) && dalloc(&s->h2, R * 128) && dalloc(&s->mask, RK) &&
      dalloc(&s->ze2, RK * 64) && dalloc(&s->out, R * 8) &&
      dalloc(&s->part, (size_t)kSplitCap * 128 * 128) && dalloc(&s->loss_part, R * 8 / 256 + 1) &&
      dalloc(&s->list, (size_t)max_envs) && dalloc(&s->list_len, 1) &&
      dalloc(&s->pbfT, kTransposed) && dalloc(&s->err, 4) && dalloc(&s->edgec, RK * 16) &&
      dalloc(&s->epos, RK) && dalloc(&s->emap, RK) &&
      dalloc(&s->escan, RK / sur::kScanBlock + 1) && dalloc(&s->etotal, 1) &&
      cudaHostAlloc((void **)&s->h_total, sizeof(int), cudaHostAllocDefault) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_sur(s);
    return fail(VMAS_ENOMEM, "cudaMalloc failed while creating the surrogate");
  }
  cudaError_t e = cudaMemset(s->p32, 0, kSurParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->pbf, 0, kSurParams * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, kSurParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, kSurParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(s->pbfT, 0, kTransposed * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMemset(s->err, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    free_sur(s);
    return cuda_fail(e, "surrogate init");
  }
  *out = s;
  return VMAS_OK;
}

int vmas_sur_destroy(vmas_surrogate *s) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  free_sur(s);
  return VMAS_OK;
}

int vmas_sur_set_params(vmas_surrogate *s, const float *h_params) {
  if (!s || !h_params) return fail(VMAS_EINVAL, "surrogate or h_params is NULL");
  for (int q = 0; q < kSurParams; ++q)
    if (!std::isfinite(h_params[q])) return fail(VMAS_EINVAL, "a parameter is not finite");
  VMAS_CUDA(cudaMemcpy(s->p32, h_params, kSurParams * sizeof(float), cudaMemcpyHostToDevice));
  f32_to_bf16_kernel<<<blocks_for(kSurParams, 256), 256>>>(s->p32, s->pbf, kSurParams);
  VMAS_CUDA(cudaGetLastError());
  if (int rc = refresh_transposed(s, nullptr)) return rc;
  VMAS_CUDA(cudaMemset(s->adam_m, 0, kSurParams * sizeof(float)));
  VMAS_CUDA(cudaMemset(s->adam_v, 0, kSurParams * sizeof(float)));
  VMAS_CUDA(cudaDeviceSynchronize());
  s->adam_t = 0;
  return VMAS_OK;
}

int vmas_sur_get_params(vmas_surrogate *s, float *h_params) {
  if (!s || !h_params) return fail(VMAS_EINVAL, "surrogate or h_params is NULL");
  VMAS_CUDA(cudaDeviceSynchronize());
  VMAS_CUDA(cudaMemcpy(h_params, s->p32, kSurParams * sizeof(float), cudaMemcpyDeviceToHost));
  return VMAS_OK;
}

int vmas_sur_set_mode(vmas_surrogate *s, int32_t mode) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  if (mode != VMAS_SUR_FUSED && mode != VMAS_SUR_LAYERED) return fail(VMAS_EINVAL, "unknown mode");
  s->mode = mode;
  return VMAS_OK;
}

int vmas_sur_forward(vmas_surrogate *s, vmas_world *w, const float *d_actions, float *d_out,
                     void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if (s->mode == VMAS_SUR_FUSED && w->sur_layout == 1)
    return sur_fused(s, w, d_actions, d_out ? d_out : s->out, false, 0.f, st);
  if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
  if (d_out && w->E)
    VMAS_CUDA(cudaMemcpyAsync(d_out, s->out, (size_t)w->E * nodes_of(w) * 8 * sizeof(float),
                              cudaMemcpyDeviceToDevice, st));
  return VMAS_OK;
}

int vmas_sur_loss_grad(vmas_surrogate *s, vmas_world *w, const float *d_actions,
                       const float *d_target, float *d_loss, float *d_grad, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  if (w->E > 0 && !d_target) return fail(VMAS_EINVAL, "d_target is NULL");
  if ((rc = ensure_training(s))) return rc;
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_forward(s, w, d_actions, true, st))) return rc;
  if ((rc = sur_backward(s, w->E, nodes_of(w), target_width(w), d_target, d_loss, st))) return rc;
  if (d_grad)
    VMAS_CUDA(cudaMemcpyAsync(d_grad, s->grad, kSurParams * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
  return VMAS_OK;
}

int vmas_sur_adam(vmas_surrogate *s, float lr, const float *d_grad, void *stream) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  if (!(lr >= 0) || !std::isfinite(lr)) return fail(VMAS_EINVAL, "lr must be >= 0");
  cudaStream_t st = as_stream(stream);
  if (d_grad && d_grad != s->grad)
    VMAS_CUDA(cudaMemcpyAsync(s->grad, d_grad, kSurParams * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
  return sur_adam(s, lr, st);
}

// Forward on the world's current state, the plain step (the world advances)
// as the target, loss and gradient into s->grad.
static int sur_train_grad(vmas_surrogate *s, vmas_world *w, const float *d_actions,
                          float *d_loss, cudaStream_t st) {
  int rc = ensure_training(s);
  if (rc) return rc;
  const int E = w->E, nodes = nodes_of(w), tw = target_width(w), R = E * nodes;
  if (E == 0) {
    VMAS_CUDA(cudaMemsetAsync(s->grad, 0, kSurParams * sizeof(float), st));
    if (d_loss) VMAS_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
    return VMAS_OK;
  }
  const size_t EN = (size_t)E * w->N;
  if ((rc = sur_forward(s, w, d_actions, true, st))) return rc;
  sur::save_nodes_kernel<<<blocks_for(R, 256), 256, 0, st>>>(E, w->N, nodes, w->planes, EN, s->save);
  VMAS_CUDA(cudaGetLastError());
  StepParams p = make_params(w);
  p.actions = d_actions;
  if ((rc = launch_step(p, st))) return rc;
  sur::targets_kernel<<<blocks_for(R, 256), 256, 0, st>>>(E, w->N, nodes, tw, w->planes, EN, s->save,
                                                           s->target);
  VMAS_CUDA(cudaGetLastError());
  return sur_backward(s, E, nodes, tw, s->target, d_loss, st);
}

int vmas_sur_train_grad(vmas_surrogate *s, vmas_world *w, const float *d_actions, float *d_loss,
                        float *d_grad, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_train_grad(s, w, d_actions, d_loss, st))) return rc;
  if (d_grad)
    VMAS_CUDA(cudaMemcpyAsync(d_grad, s->grad, kSurParams * sizeof(float), cudaMemcpyDeviceToDevice,
                              st));
  return VMAS_OK;
}

int vmas_sur_train_step(vmas_surrogate *s, vmas_world *w, const float *d_actions, float lr,
                        float *d_loss, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  if (!(lr >= 0) || !std::isfinite(lr)) return fail(VMAS_EINVAL, "lr must be >= 0");
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_train_grad(s, w, d_actions, d_loss, st))) return rc;
  if (w->E == 0) return VMAS_OK;
  return sur_adam(s, lr, st);
}

int vmas_sur_step(vmas_surrogate *s, vmas_world *w, const float *d_actions, float limit,
                  int32_t *d_n_fallback, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  if (!(limit >= 0) || !std::isfinite(limit)) return fail(VMAS_EINVAL, "limit must be >= 0");
  cudaStream_t st = as_stream(stream);
  const int E = w->E;
  if (E == 0) {
    if (d_n_fallback) VMAS_CUDA(cudaMemsetAsync(d_n_fallback, 0, sizeof(int32_t), st));
    return VMAS_OK;
  }
  VMAS_CUDA(cudaMemsetAsync(s->list_len, 0, sizeof(int), st));
  if (s->mode == VMAS_SUR_FUSED && w->sur_layout == 1) {
    if ((rc = sur_fused(s, w, d_actions, nullptr, true, limit, st))) return rc;
  } else if (w->sur_layout == 2) {
    if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
    sur::PredictBoxArgs a{};
    const size_t EN = (size_t)E * w->N;
    a.E = E; a.N = w->N;
    a.px = w->planes; a.py = w->planes + EN; a.vx = w->planes + 2 * EN; a.vy = w->planes + 3 * EN;
    a.th = w->planes + 4 * EN; a.om = w->planes + 5 * EN;
    a.param = w->param; a.out = s->out; a.limit = limit;
    a.list = s->list; a.list_len = s->list_len;
    sur::predict_box_kernel<<<blocks_for(E, sur::kPbWarps), sur::kPbWarps * 32, 0, st>>>(a);
    VMAS_CUDA(cudaGetLastError());
  } else {
    if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
    sur::PredictArgs a{};
    const size_t EN = (size_t)E * w->N;
    a.E = E; a.N = w->N;
    a.px = w->planes; a.py = w->planes + EN; a.vx = w->planes + 2 * EN; a.vy = w->planes + 3 * EN;
    a.param = w->param; a.out = s->out; a.limit = limit;
    a.list = s->list; a.list_len = s->list_len;
    sur::predict_kernel<<<blocks_for(E, sur::kPbWarps), sur::kPbWarps * 32, 0, st>>>(a);
    VMAS_CUDA(cudaGetLastError());
  }
  // the plain step for the listed envs (grid sized for all; blocks past the
  // device-side count return at once)
  StepParams p = make_params(w);
  p.actions = d_actions;
  p.env_list = s->list;
  p.env_count = s->list_len;
  if ((rc = launch_step(p, st))) return rc;
  if (d_n_fallback)
    VMAS_CUDA(cudaMemcpyAsync(d_n_fallback, s->list_len, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return VMAS_OK;
}

int vmas_sur_debug_features(vmas_surrogate *s, vmas_world *w, const float *d_actions,
                            uint16_t *d_node, uint16_t *d_edge, float *d_mask, void *stream) {
  int rc = sur_check(s, w, d_actions);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if ((rc = sur_forward(s, w, d_actions, false, st))) return rc;
  const size_t R = (size_t)w->E * nodes_of(w), RK = R * sur::kK;
  if (!R) return VMAS_OK;
  if (d_node) VMAS_CUDA(cudaMemcpyAsync(d_node, s->node, R * 16 * 2, cudaMemcpyDeviceToDevice, st));
  if (d_edge) VMAS_CUDA(cudaMemcpyAsync(d_edge, s->edge, RK * 16 * 2, cudaMemcpyDeviceToDevice, st));
  if (d_mask) VMAS_CUDA(cudaMemcpyAsync(d_mask, s->mask, RK * 4, cudaMemcpyDeviceToDevice, st));
  return VMAS_OK;
}

int vmas_debug_gemm_bf16(int32_t trans_a, int32_t trans_b, int32_t M, int32_t N, int32_t K,
                         const uint16_t *d_a, int32_t lda, const uint16_t *d_b, int32_t ldb,
                         const float *d_bias, int32_t gelu, float *d_out_f32, uint16_t *d_out_bf16,
                         int32_t splits, void *stream) {
  if (M < 0 || N < 0 || K < 0 || splits < 1 || splits > kSplitCap)
    return fail(VMAS_EINVAL, "bad GEMM sizes");
  if (splits > 1 && (d_bias || d_out_bf16 || gelu))
    return fail(VMAS_EINVAL, "split-K GEMMs take no bias, GELU or bfloat16 output");
  if ((size_t)M * N == 0) return VMAS_OK;
  if ((K > 0 && (!d_a || !d_b)) || (!d_out_f32 && !d_out_bf16))
    return fail(VMAS_EINVAL, "NULL buffer");
  if (lda < (trans_a ? M : K) || ldb < (trans_b ? K : N))
    return fail(VMAS_EINVAL, "leading dimension too small");
  cudaStream_t st = as_stream(stream);
  float *part = nullptr;
  int *err = nullptr;
  if (splits > 1) VMAS_CUDA(cudaMalloc(&part, (size_t)splits * M * N * sizeof(float)));
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(part);
    cudaFree(err);
    return fail(VMAS_ENOMEM, "GEMM error word");
  }
  int rc = gemm(st, trans_a, trans_b, M, N, K, reinterpret_cast<const bf16 *>(d_a), lda,
                reinterpret_cast<const bf16 *>(d_b), ldb, d_bias, gelu ? 1 : 0, d_out_f32, N,
                reinterpret_cast<bf16 *>(d_out_bf16), N, part, splits, err);
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    if (rc == VMAS_OK) rc = cuda_fail(cudaGetLastError(), "GEMM");
  } else if (h_err && rc == VMAS_OK) {
    rc = fail(VMAS_EDEVICE, "GEMM device error word set (bits " + std::to_string(h_err) + ")");
  }
  cudaFree(part);
  cudaFree(err);
  return rc;
}

int vmas_debug_gemm_engine(int32_t engine, int64_t *tc_launches) {
  if (engine != -1 && engine != 0 && engine != 1)
    return fail(VMAS_EINVAL, "engine must be -1, 0 or 1");
  if (engine >= 0) g_gemm_engine = engine;
  if (tc_launches) *tc_launches = g_tc_launches.load();
  return VMAS_OK;
}

int vmas_debug_gemm_timeout(int32_t on) {
  g_tc_timeout_test = on ? 1 : 0;
  return VMAS_OK;
}

int vmas_sur_check(vmas_surrogate *s, void *stream, int32_t *bits) {
  if (!s) return fail(VMAS_EINVAL, "surrogate is NULL");
  cudaStream_t st = as_stream(stream);
  int h = 0;
  VMAS_CUDA(cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  VMAS_CUDA(cudaStreamSynchronize(st));
  if (bits) *bits = h;
  if (h) {
    VMAS_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), st));
    VMAS_CUDA(cudaStreamSynchronize(st));
    return fail(VMAS_EDEVICE, "surrogate device error word set (bits " + std::to_string(h) + ")");
  }
  return VMAS_OK;
}

}  // extern "C"
