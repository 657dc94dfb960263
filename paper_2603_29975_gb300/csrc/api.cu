// C ABI of libozk (declared in include/ozk.h): handle, workspace, TMA descriptors, and the
// host-side drivers of the emulated ZGEMM and of the block-LU tau_00 solve.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ozk_params.cuh"

namespace ozk {

// --------------------------------------------------------------------- plumbing
static thread_local char g_msg[512] = "";
static thread_local uint64_t g_launches = 0;

void record_launch() { ++g_launches; }

ozk_status_t set_error(ozk_status_t st, const char* msg) {
  std::snprintf(g_msg, sizeof(g_msg), "%s", msg);
  return st;
}

ozk_status_t cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return OZK_OK;
  std::snprintf(g_msg, sizeof(g_msg), "%s: %s", what, cudaGetErrorString(e));
  return OZK_ERR_CUDA;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// 3-D fp16 map over [planes][rows][kdim] (row pitch kpad elements), box {16, box_rows, box_planes}
static ozk_status_t make_slice_map(CUtensorMap* map, void* base, long long kdim, long long kpad, long long rows,
                                   long long planes, int box_rows, int box_planes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error(OZK_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(kdim), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(planes)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(kpad) * 2, static_cast<cuuint64_t>(rows) * kpad * 2};
  cuuint32_t box[3] = {16u, static_cast<cuuint32_t>(box_rows), static_cast<cuuint32_t>(box_planes)};
  cuuint32_t es[3] = {1u, 1u, 1u};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char m[160];
    std::snprintf(m, sizeof(m), "cuTensorMapEncodeTiled failed (%d) dims %lld %lld %lld", static_cast<int>(r), kdim, rows, planes);
    return set_error(OZK_ERR_CUDA, m);
  }
  return OZK_OK;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace ozk

using namespace ozk;

// Per-kernel-kind launch profiler: CUDA events recorded on the handle's stream around each
// launch while enabled, with the algorithmic flops and bytes of that launch.
struct ProfRec { int kind; cudaEvent_t a, b; double flops, bytes, moved; };

struct ozk_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  int* d_status = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool prof = false;
  std::vector<ProfRec> recs;
  double prof_moved[OZK_KERNEL_KINDS] = {};    // bytes moved per kind at the last ozk_profile_end
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  // device copies of the host size lists of batched calls, kept by content for the life of
  // the handle (see size_table)
  std::map<std::vector<int>, int*> tables;
  // slice-count selector: [parameters | Adam first moments | second moments | gradient]
  float* sel_p = nullptr;
  int sel_t = 0;
  bool sel_ready = false;
  double sel_tol = 1e-10, sel_margin = 0.6;
  int sel_flags = 0;
  uint64_t sel_seed = 0x5E1EC7ull, sel_calls = 0;
  void* sel_ws = nullptr;                   // selector scratch (features, probes, products)
  size_t sel_ws_bytes = 0;
  ozk_selector_info sel_last{};
  // panel and leaf widths (W, w) chosen by the autotuners, keyed by (sizes..., b, S)
  std::map<std::vector<int>, std::pair<int, int>> tuned_nb;
  // side stream of the batched solve (operand splits that overlap the pivot-block inverses)
  // and the events that fork it from and join it to the handle's stream
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_join3 = nullptr;           // the side stream's split of a panel's deferred-update U rows
  long long stall_next = 0;                 // ozk_debug_stall_next_gemm: budget for the next launch
  // selector training-data log (ozk_selector_log_begin): DEVICE rows of features and targets
  float* sel_log_f = nullptr;
  float* sel_log_t = nullptr;
  int sel_log_cap = 0, sel_log_n = 0;
  void* sel_log_ws = nullptr;               // reference and trial products of the logged GEMMs
  void** one_ptrs = nullptr;                // DEVICE (M, t0, tau) of a single solve run by the batched solver
  SelDefer* sel_rec = nullptr;              // DEVICE record of the batched call's sampled checks
  size_t sel_log_ws_bytes = 0;
};

namespace {
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

cudaEvent_t prof_event(ozk_context* h) {
  if (h->pool_used == h->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->pool.push_back(e);
  }
  return h->pool[h->pool_used++];
}

// RAII scope: records a start event before and a stop event after the launches in its body.
// Launches enqueued while the stream is being captured are not timed (they run later, as graph
// nodes).
// `bytes` is the launch's algorithmic byte count; `moved` (negative: the same) the bytes its
// kernels read and write in this library's storage layout.
struct Prof {
  ozk_context* h; int kind; double flops, bytes, moved; cudaStream_t st; cudaEvent_t a = nullptr; bool on = false;
  Prof(ozk_context* hh, int k, double f, double by, cudaStream_t s = nullptr, double mv = -1.0)
      : h(hh), kind(k), flops(f), bytes(by), moved(mv < 0 ? by : mv), st(s ? s : hh->stream) {
    if (h->prof && !capturing(st)) { on = true; a = prof_event(h); cudaEventRecord(a, st); }
  }
  ~Prof() {
    if (on) {
      cudaEvent_t b = prof_event(h);
      cudaEventRecord(b, st);
      h->recs.push_back({kind, a, b, flops, bytes, moved});
    }
  }
};
}  // namespace

// --------------------------------------------------------------------- workspace
static ozk_status_t ensure_ws(ozk_context* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return OZK_OK;
  if (capturing(h->stream))
    return set_error(OZK_ERR_CAPTURE, "workspace must grow during stream capture: call ozk_reserve first");
  ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  size_t nb = align_up(bytes + (bytes >> 3), 1 << 20);
  st = cuda_check(cudaMalloc(&h->ws, nb), "cudaMalloc(workspace)");
  if (st) return st;
  st = cuda_check(cudaMemset(h->ws, 0, nb), "cudaMemset(workspace)");
  if (st) return st;
  h->ws_bytes = nb;
  return OZK_OK;
}

// Device copy of a host size list of a batched call.  Lists are kept by content for the life of
// the handle, so a launch captured into a CUDA graph keeps reading a table that later calls
// never overwrite, and a repeated call uploads nothing.  A list first seen while the stream is
// being captured is an error: neither the allocation nor the upload of a pageable host array can
// be captured, so one call with the same sizes has to come before the capture.  Past
// kMaxTables distinct lists the cache is emptied (after synchronising the stream), which
// invalidates graphs captured before.
constexpr size_t kMaxTables = 4096;

// room for k more tables before a function takes several: a cache flush in the middle would
// free the tables it already holds
static ozk_status_t table_room(ozk_context* h, size_t k) {
  if (h->tables.size() + k <= kMaxTables) return OZK_OK;
  if (capturing(h->stream)) return set_error(OZK_ERR_CAPTURE, "size-table cache full during stream capture");
  ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  for (auto& kv : h->tables) cudaFree(kv.second);
  h->tables.clear();
  return OZK_OK;
}

static ozk_status_t size_table(ozk_context* h, std::vector<int>&& key, const int** out) {
  auto it = h->tables.find(key);
  if (it != h->tables.end()) { *out = it->second; return OZK_OK; }
  if (capturing(h->stream))
    return set_error(OZK_ERR_CAPTURE, "batched sizes first seen during stream capture: make one call with the "
                                      "same sizes before capturing");
  if (h->tables.size() >= kMaxTables) {
    ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (st) return st;
    for (auto& kv : h->tables) cudaFree(kv.second);
    h->tables.clear();
  }
  int* d = nullptr;
  const size_t bytes = std::max<size_t>(1, key.size()) * sizeof(int);
  ozk_status_t st = cuda_check(cudaMalloc(&d, bytes), "cudaMalloc(size table)");
  if (st) return st;
  st = cuda_check(cudaMemcpyAsync(d, key.data(), key.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream),
                  "upload size table");
  if (st) { cudaFree(d); return st; }
  *out = d;
  h->tables.emplace(std::move(key), d);
  return OZK_OK;
}

// --------------------------------------------------------------------- emulated GEMM core
namespace {

struct OpFlags { int trans, conj; };
constexpr int PAIRS_DIAG = 2;                        // internal pair mode of the Ozaki-II products
bool parse_op(char c, OpFlags* f) {
  switch (c) {
    case 'N': case 'n': f->trans = 0; f->conj = 0; return true;
    case 'T': case 't': f->trans = 1; f->conj = 0; return true;
    case 'C': case 'c': f->trans = 1; f->conj = 1; return true;
    default: return false;
  }
}

// Problem description for one (possibly batched) emulated GEMM.  Either the single fields
// are used (batch == 1, tables == nullptr) or device tables of `batch` entries.
struct EmuGemm {
  OpFlags oa, ob;
  int batch = 1;
  int mmax = 0, nmax = 0, kmax = 0;          // host-known maxima
  // single problem
  const double2* A = nullptr; int lda = 0; const double2* B = nullptr; int ldb = 0;
  double2* C = nullptr; int ldc = 0; int m = 0, n = 0, k = 0;
  // device tables (batched)
  const double2* const* tA = nullptr; const int* tlda = nullptr;
  const double2* const* tB = nullptr; const int* tldb = nullptr;
  double2* const* tC = nullptr; const int* tldc = nullptr;
  const int* tm = nullptr; const int* tn = nullptr; const int* tk = nullptr;
  double ar = 1, ai = 0, br = 0, bi = 0;
  int S = 7, pair_mode = OZK_PAIRS_TRI;
  int mode = -1;                             // -1: derive from alpha/beta
  long long* groups = nullptr;               // group dump (test hook)
  int16_t* dbg_digits_a = nullptr; int* dbg_exps_a = nullptr;
  int skm = 0, skn = 0;                        // skip box (single problem)
  const int* tskm = nullptr; const int* tskn = nullptr;   // skip box tables (batched)
  int box_m = 0, box_n = 0;                   // batched: smallest skip box over the problems
  double sum_mnk = -1;                        // sum over problems of m n k (batched; -1: single)
  double sum_mk = 0, sum_nk = 0;              // operand sizes (complex elements) for byte counts
  long long zsA = 0, zsB = 0;                 // uniform batch of single-size problems: operand strides
  // Ozaki-II (pair_mode PAIRS_DIAG): residue planes of beta-bit integer images, products added
  // to the int32 buffer resid (row pitch ldres)
  const Oz2Tables* oz2 = nullptr; int beta = 0; int* resid = nullptr; long long ldres = 0;
  double2* const* crow = nullptr; int crow_b = 0;   // row-block scatter of the output
  const int* crow_n = nullptr;                // per-output order (device), or none
  const int* crow_perm = nullptr;             // row block a of the plane -> output crow_perm[a]
  // remapped GEMM problems over the split planes of a uniform batch: problem z (of gbatch)
  // multiplies rows [remap[2z + 1], + gm[z]) of plane remap[2z] by its first gn[z] columns
  const int* remap = nullptr; int gbatch = 0; const int* gm = nullptr; const int* gn = nullptr;
  // partial runs: split only the operands in split_sides (1: A, 2: B, 3: both; an operand left
  // out must already be split into this workspace by an earlier run of the same problem), and
  // the slice GEMM only if run_gemm; on `stream` (nullptr: the handle's stream)
  int split_sides = 3;
  bool run_gemm = true;
  bool ksplit_ok = false;                     // split K allowed (a whole-workspace single GEMM call)
  cudaStream_t stream = nullptr;
};

struct GemmPlan {
  int G, BN, maxpairs, npairs, kpad, rowsA, rowsB, nstage, chunk_kb, kblocks, magic;
  int ksplit;                                 // split-K units per tile (single problems with few tiles)
  size_t offA, offB, offE, offF, offT, offP, offGA, offGB, total;
};

ozk_status_t plan_gemm(const EmuGemm& g, GemmPlan* P) {
  const int S = g.S;
  if (S < 1 || S > 16) return set_error(OZK_ERR_ARG, "S must be in 1..16");
  const bool full = g.pair_mode == OZK_PAIRS_FULL;
  const bool diag = g.pair_mode == PAIRS_DIAG;          // Ozaki-II: one product per modulus
  P->G = full ? 2 * S - 1 : S;
  if (P->G > 16) return set_error(OZK_ERR_ARG, "full pair mode supports S <= 8");
  P->BN = P->G <= 8 ? 64 : 32;
  P->maxpairs = diag ? 1 : S;
  P->npairs = diag ? S : (full ? S * S : S * (S + 1) / 2);
  const long long kp2 = 2LL * g.kmax;
  P->kpad = static_cast<int>(align_up(static_cast<size_t>(std::max<long long>(kp2, 16)), 8));
  P->rowsA = std::max(g.mmax, 1);
  P->rowsB = 2 * std::max(g.nmax, 1);
  const size_t stage = static_cast<size_t>(S) * (128 + P->BN) * 32;
  P->nstage = static_cast<int>(std::min<size_t>(6, (200 * 1024 - 2048) / stage));
  if (P->nstage < 1) return set_error(OZK_ERR_ARG, "S too large for the shared-memory pipeline");
  P->kblocks = static_cast<int>((kp2 + 15) / 16);
  // exactness chunk: every product of two digits is <= 2^14 in magnitude; an FP32 accumulator
  // stays exact up to 2^24 (1024 terms) and allows the one-add conversion below 2^22 (255 terms)
  const int kb_magic = 255 / (16 * P->maxpairs);
  if (kb_magic >= 1 && P->kblocks <= kb_magic) { P->chunk_kb = P->kblocks; P->magic = 1; }
  else { P->chunk_kb = std::max(1, 64 / P->maxpairs); P->magic = 0; }
  // exact 128-bit sum: 8 (G - 1) weight bits + 14 product bits + log2(terms) + sign
  double terms = static_cast<double>(kp2) * P->maxpairs + 1.0;
  int need = 8 * (P->G - 1) + 14 + static_cast<int>(std::ceil(std::log2(terms))) + 2;
  // the integer group dump (test hook) never forms the 128-bit sum
  if (need > 127 && g.mode != EPI_GROUPS && g.mode != EPI_RESIDUES)
    return set_error(OZK_ERR_RANGE, "exact 128-bit reconstruction could overflow for this S and k");
  size_t off = 0;
  P->offA = off; off = align_up(off + static_cast<size_t>(g.batch) * S * P->rowsA * P->kpad * 2, 1024);
  P->offB = off; off = align_up(off + static_cast<size_t>(g.batch) * S * P->rowsB * P->kpad * 2, 1024);
  P->offE = off; off = align_up(off + static_cast<size_t>(g.batch) * P->rowsA * 4, 256);
  P->offF = off; off = align_up(off + static_cast<size_t>(g.batch) * std::max(g.nmax, 1) * 4, 256);
  P->offT = off;                                                     // tile prefix sums
  off = align_up(off + (static_cast<size_t>(std::max(g.batch, g.gbatch)) + 1) * 4, 256);
  // row maxima of the K-parallel split (left, right operand)
  P->offGA = off; off = align_up(off + static_cast<size_t>(g.batch) * P->rowsA * 8, 256);
  P->offGB = off; off = align_up(off + static_cast<size_t>(g.batch) * std::max(g.nmax, 1) * 8, 256);
  // split K: a single problem whose tiles fill less than half of the SMs and whose K spans
  // several exactness chunks runs up to 8 units per tile, each over a share of the chunks,
  // whose exact partial sums (two int64 per stacked output) a finishing kernel adds and rounds;
  // for the 128-bit epilogue of the triangular schedules on 64-column tiles (store, LU and
  // general modes)
  P->ksplit = 1;
  P->offP = off;
  {
    const double terms = 16.0 * P->kblocks * P->maxpairs;
    const int bits = static_cast<int>(std::ceil(std::log2(terms))) + 14 + 8 * (P->G - 1) + 1;
    const bool fit64 = P->G <= 5 && bits <= 63;
    const bool modes = g.mode < 0 || g.mode == EPI_STORE || g.mode == EPI_LU || g.mode == EPI_GENERAL;
    if (g.ksplit_ok && g.batch == 1 && g.tm == nullptr && !g.remap && !g.crow && !diag && g.pair_mode == OZK_PAIRS_TRI &&
        P->BN == 64 && P->G <= 8 && !fit64 && modes && g.m > 0 && g.n > 0) {
      const int nch = (P->kblocks + P->chunk_kb - 1) / P->chunk_kb;
      const long long tiles = static_cast<long long>((g.m + 127) / 128) * ((2LL * g.n + 63) / 64);
      const int sms = gpu_sm_count();
      if (nch >= 2 && 2 * tiles <= sms)
        P->ksplit = static_cast<int>(std::min<long long>({static_cast<long long>(nch), sms / tiles, 8LL}));
    }
    if (P->ksplit > 1) off = align_up(off + static_cast<size_t>(P->ksplit) * 2 * g.n * g.m * sizeof(long long) * 2, 256);
  }
  P->total = off;
  return OZK_OK;
}

ozk_status_t run_emulated(ozk_context* h, const EmuGemm& g, size_t ws_offset = 0) {
  GemmPlan P;
  ozk_status_t st = plan_gemm(g, &P);
  if (st) return st;
  st = ensure_ws(h, ws_offset + P.total);
  if (st) return st;
  uint8_t* ws = static_cast<uint8_t*>(h->ws) + ws_offset;
  __half* As = reinterpret_cast<__half*>(ws + P.offA);
  __half* Bs = reinterpret_cast<__half*>(ws + P.offB);
  int* e = reinterpret_cast<int*>(ws + P.offE);
  int* f = reinterpret_cast<int*>(ws + P.offF);
  const bool single = g.tm == nullptr;
  const int S = g.S;
  cudaStream_t stream = g.stream ? g.stream : h->stream;

  const bool diag = g.pair_mode == PAIRS_DIAG;
  SplitParams sp{};
  sp.S = S; sp.nbits = diag ? g.beta : 8 * S - 1; sp.status = h->d_status; sp.kpad = P.kpad;
  // left operand: rows of op(A); logical X[r][l] = op(A)[r][l]
  sp.trans = g.oa.trans; sp.conj = g.oa.conj; sp.side = 0;
  sp.out_rows = P.rowsA; sp.out = As; sp.exps = e; sp.exp_stride = P.rowsA;
  sp.dbg_digits = g.dbg_digits_a;
  sp.gmax = reinterpret_cast<unsigned long long*>(ws + P.offGA);
  sp.kgroups = 1;
  if (single) { sp.X = nullptr; sp.X1 = g.A; sp.ld1 = g.lda; sp.rows1 = g.m; sp.k1 = g.k; sp.zstride1 = g.zsA; }
  else { sp.X = g.tA; sp.ld = g.tlda; sp.rows = g.tm; sp.kdim = g.tk; }
  const double smnk = g.sum_mnk >= 0 ? g.sum_mnk : static_cast<double>(g.m) * g.n * g.k;
  const double smk = g.sum_mnk >= 0 ? g.sum_mk : static_cast<double>(g.m) * g.k;
  const double snk = g.sum_mnk >= 0 ? g.sum_nk : static_cast<double>(g.n) * g.k;
  // right operand: columns of op(B); logical X[j][l] = op(B)[l][j]
  SplitParams sq = sp;
  sq.trans = g.ob.trans ? 0 : 1; sq.conj = g.ob.conj; sq.side = 1;
  sq.out_rows = P.rowsB; sq.out = Bs; sq.exps = f; sq.exp_stride = std::max(g.nmax, 1);
  sq.dbg_digits = nullptr;
  sq.gmax = reinterpret_cast<unsigned long long*>(ws + P.offGB);
  if (single) { sq.X = nullptr; sq.X1 = g.B; sq.ld1 = g.ldb; sq.rows1 = g.n; sq.k1 = g.k; sq.zstride1 = g.zsB; }
  else { sq.X = g.tB; sq.ld = g.tldb; sq.rows = g.tn; sq.kdim = g.tk; }
  const bool split_a = (g.split_sides & 1) != 0, split_b = (g.split_sides & 2) != 0;
  if (split_a || split_b) {
    // algorithmic bytes (int8 digits): read 16 per complex element, write 2S (left operand: Re,
    // Im) or 3S (right operand: Re, Im, -Im); moved: the fp16 planes written here, S x 2 x 2
    // (left) or S x 4 x 2 (right, two stacked rows per column)
    Prof pr(h, OZK_KIND_SPLIT, 0.0, (split_a ? smk * (16.0 + 2.0 * S) : 0.0) + (split_b ? snk * (16.0 + 3.0 * S) : 0.0),
            stream, (split_a ? smk * (16.0 + 4.0 * S) : 0.0) + (split_b ? snk * (16.0 + 8.0 * S) : 0.0));
    if (diag) {
      if (split_a) launch_residue_split(sp, *g.oz2, g.mmax, g.batch, stream);
      if (split_b) launch_residue_split(sq, *g.oz2, g.nmax, g.batch, stream);
    } else if (split_a && split_b) {
      launch_split(sp, g.mmax, &sq, g.nmax, g.kmax, g.batch, stream);
    } else if (split_a) {
      launch_split(sp, g.mmax, nullptr, 0, g.kmax, g.batch, stream);
    } else {
      launch_split(sq, g.nmax, nullptr, 0, g.kmax, g.batch, stream);
    }
  }
  if (!g.run_gemm) return cuda_check(cudaGetLastError(), "split launch");

  CUtensorMap ta, tb;
  st = make_slice_map(&ta, As, 2LL * g.kmax, P.kpad, P.rowsA, static_cast<long long>(S) * g.batch, 128, S);
  if (st) return st;
  st = make_slice_map(&tb, Bs, 2LL * g.kmax, P.kpad, P.rowsB, static_cast<long long>(S) * g.batch, P.BN, S);
  if (st) return st;

  GemmParams gp{};
  gp.S = S; gp.ngroups = P.G; gp.kblocks = P.kblocks; gp.chunk_kb = P.chunk_kb; gp.nstage = P.nstage;
  gp.magic = P.magic;
  {
    // group g receives the products of its own pairs only: 16 per K-block and pair, each at most
    // 2^14 in magnitude, so a group of np pairs stays within 2^22 when 16 np chunk_kb <= 256
    int np[32] = {0};
    for (int s1 = 1; s1 <= S; ++s1)
      for (int t1 = 1; t1 <= S; ++t1) {
        if (diag && s1 != t1) continue;
        if (!diag && g.pair_mode != OZK_PAIRS_FULL && s1 + t1 > S + 1) continue;
        const int gi = diag ? s1 - 1 : s1 + t1 - 2;
        if (gi < 32) ++np[gi];
      }
    gp.magic_mask = 0;
    for (int gi = 0; gi < std::min(P.G, 32); ++gi)
      if (np[gi] > 0 && 16LL * np[gi] * P.chunk_kb <= 256) gp.magic_mask |= static_cast<int>(1u << gi);
  }
  {
    // the 64-bit epilogue: |sum| < 2^(ceil(log2 terms) + 14 + 8 (G - 1) + 1) <= 2^63, terms = the
    // digit products one group receives over all its exactness chunks
    const double terms = 16.0 * P.kblocks * P.maxpairs;
    const int bits = static_cast<int>(std::ceil(std::log2(terms))) + 14 + 8 * (P.G - 1) + 1;
    gp.fit64 = (P.G <= 5 && bits <= 63) ? 1 : 0;
  }
  gp.fullset = g.pair_mode == OZK_PAIRS_FULL ? 1 : 0;
  const int gmax = (g.pair_mode == OZK_PAIRS_FULL) ? 2 * S : S + 1;
  gp.base_exp = -2 * (8 * S - 1) + 8 * (2 * S - gmax);
  gp.diag_pairs = diag ? 1 : 0;
  gp.stall_cycles = h->stall_next;
  h->stall_next = 0;
  gp.resid = g.resid; gp.ldres = g.ldres;
  gp.ar = g.ar; gp.ai = g.ai; gp.br = g.br; gp.bi = g.bi;
  if (g.mode >= 0) gp.mode = g.mode;
  else if (g.br == 0.0 && g.bi == 0.0) gp.mode = 0;
  else if (g.ar == -1.0 && g.ai == 0.0 && g.br == 1.0 && g.bi == 0.0) gp.mode = 1;
  else gp.mode = 2;
  gp.e = e; gp.f = f; gp.e_stride = P.rowsA; gp.f_stride = std::max(g.nmax, 1);
  gp.groups = g.groups; gp.status = h->d_status;
  if (single) { gp.m = nullptr; gp.m1 = g.m; gp.n1 = g.n; gp.C1 = g.C; gp.ldc1 = g.ldc; gp.skm1 = g.skm; gp.skn1 = g.skn; }
  else { gp.m = g.tm; gp.n = g.tn; gp.C = g.tC; gp.ldc = g.tldc; gp.skm = g.tskm; gp.skn = g.tskn; }
  gp.crow = g.crow; gp.crow_b = g.crow_b; gp.crow_n = g.crow_n; gp.crow_perm = g.crow_perm;
  if (g.remap) {
    gp.remap = reinterpret_cast<const int2*>(g.remap);
    gp.m = g.gm; gp.n = g.gn; gp.C = nullptr; gp.ldc = nullptr; gp.skm = gp.skn = nullptr;
  }
  gp.box_m = single ? g.skm : (g.tskm ? g.box_m : 0);
  gp.box_n = single ? g.skn : (g.tskn ? g.box_n : 0);
  int np = 0;
  if (diag) {
    for (int t = 0; t < S; ++t) {
      gp.ps[np] = gp.pt[np] = gp.pg[np] = static_cast<uint8_t>(t);
      gp.pfirst[np] = 1;
      ++np;
    }
  }
  for (int gg = 2; gg <= gmax && !diag; ++gg) {
    bool first = true;
    for (int s = 1; s <= S; ++s) {
      const int t = gg - s;
      if (t < 1 || t > S) continue;
      gp.ps[np] = static_cast<uint8_t>(s - 1);
      gp.pt[np] = static_cast<uint8_t>(t - 1);
      gp.pg[np] = static_cast<uint8_t>(gg - 2);
      gp.pfirst[np] = first ? 1 : 0;
      first = false;
      ++np;
    }
  }
  gp.npairs = np;
  const int gbatch = g.remap ? g.gbatch : g.batch;
  if (!single || g.remap) {
    // problems of different sizes: every CTA enumerates exactly the tiles of each problem
    int* tp = reinterpret_cast<int*>(ws + P.offT);
    gp.tile_prefix = tp;
    launch_tile_prefix(gp, P.BN, gbatch, tp, stream);
  }
  if (P.ksplit > 1) {
    gp.ksplit = P.ksplit;
    gp.part = reinterpret_cast<longlong2*>(ws + P.offP);
  }
  {
    // algorithmic integer ops: every pair is one real GEMM m x 2n x 2k (8 m n k); a split K's
    // finishing kernel belongs to the same product
    Prof pr(h, OZK_KIND_SLICE_GEMM, 8.0 * np * smnk, 0.0, stream);
    launch_slice_gemm(ta, tb, gp, P.BN, g.remap ? std::min(g.mmax, 128) : g.mmax, g.nmax, gbatch, stream);
    if (P.ksplit > 1) launch_finish_split(gp, stream);
  }
  return cuda_check(cudaGetLastError(), "slice GEMM launch");
}

ozk_status_t check_dims(OpFlags oa, OpFlags ob, int m, int n, int k, int lda, int ldb, int ldc) {
  if (m < 0 || n < 0 || k < 0) return set_error(OZK_ERR_ARG, "negative dimension");
  const int ra = oa.trans ? k : m, rb = ob.trans ? n : k;
  if (lda < std::max(1, ra)) return set_error(OZK_ERR_ARG, "lda too small");
  if (ldb < std::max(1, rb)) return set_error(OZK_ERR_ARG, "ldb too small");
  if (ldc < std::max(1, m)) return set_error(OZK_ERR_ARG, "ldc too small");
  return OZK_OK;
}

}  // namespace

// --------------------------------------------------------------------- slice-count selector
// Scratch of the selector, separate from the GEMM workspace (the S = 0 path runs emulated
// GEMMs while its features and probe products are alive).
static ozk_status_t ensure_sel_ws(ozk_context* h, size_t bytes) {
  if (bytes <= h->sel_ws_bytes) return OZK_OK;
  if (capturing(h->stream)) return set_error(OZK_ERR_CAPTURE, "selector scratch must grow during stream capture");
  ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  if (h->sel_ws) cudaFree(h->sel_ws);
  h->sel_ws = nullptr;
  h->sel_ws_bytes = 0;
  const size_t nb = align_up(bytes + (bytes >> 3), 1 << 20);
  st = cuda_check(cudaMalloc(&h->sel_ws, nb), "cudaMalloc(selector scratch)");
  if (st) return st;
  h->sel_ws_bytes = nb;
  return OZK_OK;
}

static ozk_status_t sel_alloc_params(ozk_context* h) {
  if (h->sel_p) return OZK_OK;
  ozk_status_t st = cuda_check(cudaMalloc(&h->sel_p, 4 * sizeof(float) * SEL_NPARAMS), "cudaMalloc(selector)");
  if (st) return st;
  return cuda_check(cudaMemset(h->sel_p, 0, 4 * sizeof(float) * SEL_NPARAMS), "cudaMemset(selector)");
}

// upload parameters, clear the Adam moments
static ozk_status_t sel_upload(ozk_context* h, const float* host) {
  ozk_status_t st = sel_alloc_params(h);
  if (st) return st;
  st = cuda_check(cudaMemcpy(h->sel_p, host, sizeof(float) * SEL_NPARAMS, cudaMemcpyHostToDevice), "upload params");
  if (st) return st;
  st = cuda_check(cudaMemset(h->sel_p + SEL_NPARAMS, 0, 3 * sizeof(float) * SEL_NPARAMS), "clear Adam state");
  if (st) return st;
  h->sel_t = 0;
  h->sel_ready = true;
  return OZK_OK;
}

struct SelScratch {
  SelVecStats a, b;
  int* ex;
  double2 *X, *yh, *yl, *zh, *zl, *Wh, *Wl, *part, *D;   // probe products as double-doubles
  float *f, *Y;
  SelAux* aux;
};

// carve the scratch of the product op(A) op(B) (m x k times k x n); D (m x n) on request
static ozk_status_t sel_scratch(ozk_context* h, int m, int n, int k, bool needD, SelScratch* s) {
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1), 256); return o; };
  const size_t P = SEL_PROBES;
  const size_t o_ar = take(8 * size_t(m)), o_ae = take(4 * size_t(m)), o_ash = take(8 * size_t(m)), o_az = take(4 * size_t(m));
  const size_t o_acr = take(8 * size_t(m));
  const size_t o_br = take(8 * size_t(n)), o_be = take(4 * size_t(n)), o_bsh = take(8 * size_t(n)), o_bz = take(4 * size_t(n));
  const size_t o_bcr = take(8 * size_t(n));
  const size_t o_ex = take(8), o_X = take(16 * P * n), o_yh = take(16 * P * k), o_yl = take(16 * P * k);
  const size_t o_zh = take(16 * P * m), o_zl = take(16 * P * m), o_Wh = take(16 * P * m), o_Wl = take(16 * P * m);
  // chunk partials of the row-strided products: y (k rows over n), zs and W (m rows over k, n)
  const size_t prow = std::max<size_t>({size_t(k) * gemv_chunks(n), size_t(m) * gemv_chunks(k),
                                        size_t(m) * gemv_chunks(n)});
  const size_t o_part = take(32 * P * prow);
  const size_t o_f = take(4 * SEL_NF), o_Y = take(4 * SEL_NO), o_aux = take(sizeof(SelAux));
  const size_t o_D = needD ? take(16 * size_t(m) * n) : 0;
  ozk_status_t st = ensure_sel_ws(h, off);
  if (st) return st;
  uint8_t* b = static_cast<uint8_t*>(h->sel_ws);
  s->a = {reinterpret_cast<double*>(b + o_ar), reinterpret_cast<int*>(b + o_ae), reinterpret_cast<double*>(b + o_ash),
          reinterpret_cast<int*>(b + o_az), reinterpret_cast<double*>(b + o_acr)};
  s->b = {reinterpret_cast<double*>(b + o_br), reinterpret_cast<int*>(b + o_be), reinterpret_cast<double*>(b + o_bsh),
          reinterpret_cast<int*>(b + o_bz), reinterpret_cast<double*>(b + o_bcr)};
  s->ex = reinterpret_cast<int*>(b + o_ex);
  s->X = reinterpret_cast<double2*>(b + o_X);
  s->yh = reinterpret_cast<double2*>(b + o_yh);
  s->yl = reinterpret_cast<double2*>(b + o_yl);
  s->zh = reinterpret_cast<double2*>(b + o_zh);
  s->zl = reinterpret_cast<double2*>(b + o_zl);
  s->Wh = reinterpret_cast<double2*>(b + o_Wh);
  s->Wl = reinterpret_cast<double2*>(b + o_Wl);
  s->part = reinterpret_cast<double2*>(b + o_part);
  s->f = reinterpret_cast<float*>(b + o_f);
  s->Y = reinterpret_cast<float*>(b + o_Y);
  s->aux = reinterpret_cast<SelAux*>(b + o_aux);
  s->D = needD ? reinterpret_cast<double2*>(b + o_D) : nullptr;
  return OZK_OK;
}

// features of op(A) op(B) into s.f, the scaled probe product into s.zs, E and ||zs||^2 into s.aux
static ozk_status_t sel_features(ozk_context* h, const OpFlags& oa, const OpFlags& ob, int m, int n, int k,
                                 const double2* A, int lda, const double2* B, int ldb, uint64_t seed,
                                 const SelScratch& s) {
  cudaStream_t st = h->stream;
  SelBases bs;
  for (int i = 0; i < 2 * SEL_PROBES; ++i) bs.b[i] = sm_base_host(seed, static_cast<uint64_t>(i));
  launch_probe(s.X, n, bs, st);
  // rows of op(A): rows of A (strided) or columns of A (contiguous)
  launch_vec_stats(A, lda, m, k, oa.trans != 0, s.a, st);
  // columns of op(B): columns of B (contiguous) or rows of B (strided)
  launch_vec_stats(B, ldb, n, k, ob.trans == 0, s.b, st);
  launch_max_exp(s.a, m, s.b, n, s.ex, st);
  // y = (2^-EB op(B)) X, zs = (2^-EA op(A)) y, both double-doubles
  launch_gemv(B, ldb, k, n, ob.trans == 0 ? 0 : (ob.conj ? 2 : 1), s.X, nullptr, n, s.yh, s.yl, s.part, s.ex, 1, st);
  launch_gemv(A, lda, m, k, oa.trans == 0 ? 0 : (oa.conj ? 2 : 1), s.yh, s.yl, k, s.zh, s.zl, s.part, s.ex, 0, st);
  launch_selector_features(s.a, m, s.b, n, k, s.X, s.zh, s.ex, s.f, s.aux, st);
  return cuda_check(cudaGetLastError(), "selector feature launches");
}

static ozk_status_t read_aux(ozk_context* h, const SelAux* d, SelAux* out) {
  ozk_status_t st = cuda_check(cudaMemcpyAsync(out, d, sizeof(SelAux), cudaMemcpyDeviceToHost, h->stream), "read aux");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
}

// Training-data row of the selector for the GEMM g (features already in s.f): the log10
// relative Frobenius errors of its products at S = 3..10 against the S = 12 product.
constexpr int SEL_SREF = 12;
static ozk_status_t sel_log_gemm(ozk_context* h, const EmuGemm& g, const SelScratch& s, size_t ws_offset) {
  const int m = g.m, n = g.n;
  const size_t prod = align_up(sizeof(double2) * static_cast<size_t>(m) * n, 256);
  const size_t need = 2 * prod + align_up(sizeof(double) * 2 * static_cast<size_t>(n), 256) + 256;
  if (need > h->sel_log_ws_bytes) {
    ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (st) return st;
    if (h->sel_log_ws) cudaFree(h->sel_log_ws);
    h->sel_log_ws = nullptr;
    h->sel_log_ws_bytes = 0;
    st = cuda_check(cudaMalloc(&h->sel_log_ws, need + (need >> 2)), "cudaMalloc(selector log scratch)");
    if (st) return st;
    h->sel_log_ws_bytes = need + (need >> 2);
  }
  uint8_t* base = static_cast<uint8_t*>(h->sel_log_ws);
  double2* ref = reinterpret_cast<double2*>(base);
  double2* trial = reinterpret_cast<double2*>(base + prod);
  double* part = reinterpret_cast<double*>(base + 2 * prod);
  double* rel = reinterpret_cast<double*>(base + 2 * prod + align_up(sizeof(double) * 2 * static_cast<size_t>(n), 256));
  const int row = h->sel_log_n++;
  ozk_status_t st = cuda_check(cudaMemcpyAsync(h->sel_log_f + static_cast<size_t>(row) * SEL_NF, s.f,
                                               sizeof(float) * SEL_NF, cudaMemcpyDeviceToDevice, h->stream),
                               "copy features");
  if (st) return st;
  EmuGemm d = g;
  d.ar = 1; d.ai = 0; d.br = 0; d.bi = 0;
  d.pair_mode = OZK_PAIRS_TRI;
  d.mode = -1;
  d.ldc = m;
  d.C = ref; d.S = SEL_SREF;
  st = run_emulated(h, d, ws_offset);
  for (int S = SEL_SMIN; S <= SEL_SMAX && !st; ++S) {
    d.C = trial; d.S = S;
    st = run_emulated(h, d, ws_offset);
    if (st) break;
    launch_rel_diff(m, n, trial, m, ref, m, part, rel, h->stream);
    launch_log_err(rel, h->sel_log_t + static_cast<size_t>(row) * SEL_NO + (S - SEL_SMIN), h->stream);
  }
  if (st) return st;
  return cuda_check(cudaGetLastError(), "selector log launches");
}

// S = 0: choose S, compute the product, check it with the probes, fall back to SMAX.  Inside a
// solve (defer != null) the check is recorded on the device instead (no second host read, no
// per-GEMM fallback: the solve is redone at SMAX when any check failed), and force_S > 0 skips
// the choice (the redone solve, still checked).
static ozk_status_t zgemm_auto(ozk_context* h, const EmuGemm& g, size_t ws_offset = 0, SelDefer* defer = nullptr,
                               int force_S = 0) {
  if (!h->sel_ready)
    return set_error(OZK_ERR_ARG, "S = 0 needs selector parameters (ozk_selector_init, _load or _set_params)");
  if (capturing(h->stream))
    return set_error(OZK_ERR_CAPTURE, "S = 0 synchronises to read the selector's choice and cannot be captured");
  const int m = g.m, n = g.n, k = g.k;
  const bool direct = g.ar == 1.0 && g.ai == 0.0 && g.br == 0.0 && g.bi == 0.0;
  SelScratch s;
  ozk_status_t st = sel_scratch(h, m, n, k, !direct, &s);
  if (st) return st;
  ozk_selector_info info{};
  info.probe_seed = h->sel_seed + h->sel_calls++;
  st = sel_features(h, g.oa, g.ob, m, n, k, g.A, g.lda, g.B, g.ldb, info.probe_seed, s);
  if (st) return st;
  if (h->sel_log_f && h->sel_log_n < h->sel_log_cap && force_S == 0) {
    st = sel_log_gemm(h, g, s, ws_offset);
    if (st) return st;
  }
  SelAux aux{};
  if (force_S > 0) {
    aux.S = force_S;
  } else {
    launch_mlp_forward(h->sel_p, s.f, 1, nullptr, nullptr, s.Y, h->stream);
    launch_choose(s.Y, static_cast<float>(std::log10(h->sel_tol) - h->sel_margin), s.aux, h->stream);
    st = read_aux(h, s.aux, &aux);
    if (st) return st;
  }
  info.S_selected = aux.S;
  for (int o = 0; o < SEL_NO; ++o) info.predicted_log10_err[o] = aux.pred[o];
  EmuGemm d = g;
  d.C = direct ? g.C : s.D;
  d.ldc = direct ? g.ldc : m;
  d.ar = 1; d.ai = 0; d.br = 0; d.bi = 0;
  d.pair_mode = OZK_PAIRS_TRI;
  auto product_and_check = [&](int S, double* r) -> ozk_status_t {
    d.S = S;
    ozk_status_t e = run_emulated(h, d, ws_offset);
    if (e) return e;
    launch_gemv(d.C, d.ldc, m, n, 0, s.X, nullptr, n, s.Wh, s.Wl, s.part, nullptr, 0, h->stream, true);
    launch_residual(s.Wh, s.Wl, s.zh, s.zl, m, s.aux, reinterpret_cast<double*>(s.part), h->stream);
    SelAux a2;
    e = read_aux(h, s.aux, &a2);
    *r = a2.resid;
    return e;
  };
  // the 4-probe estimate scatters around the true error: a product passes when its estimate is
  // at most half the tolerance
  const double pass = 0.5 * h->sel_tol;
  if (defer) {
    d.S = aux.S;
    st = run_emulated(h, d, ws_offset);
    if (st) return st;
    launch_gemv(d.C, d.ldc, m, n, 0, s.X, nullptr, n, s.Wh, s.Wl, s.part, nullptr, 0, h->stream, true);
    launch_residual(s.Wh, s.Wl, s.zh, s.zl, m, s.aux, reinterpret_cast<double*>(s.part), h->stream);
    launch_defer_check(s.aux, aux.S, force_S == 0, pass, defer, h->stream);
    if (!direct) launch_axpby(m, n, s.D, m, g.C, g.ldc, g.ar, g.ai, g.br, g.bi, h->stream);
    return cuda_check(cudaGetLastError(), "deferred check launches");
  }
  double r = 0.0;
  st = product_and_check(aux.S, &r);
  if (st) return st;
  info.residual_selected = r;
  info.S_used = aux.S;
  if (!(r <= pass) && !(h->sel_flags & OZK_SEL_NO_FALLBACK) && aux.S < SEL_SMAX) {
    st = product_and_check(SEL_SMAX, &r);
    if (st) return st;
    info.S_used = SEL_SMAX;
    info.fallback = 1;
  }
  info.residual = r;
  info.residual_ok = r <= pass ? 1 : 0;
  if (!direct) {
    launch_axpby(m, n, s.D, m, g.C, g.ldc, g.ar, g.ai, g.br, g.bi, h->stream);
    st = cuda_check(cudaGetLastError(), "axpby launch");
    if (st) return st;
  }
  h->sel_last = info;
  if (!info.residual_ok && (h->sel_flags & OZK_SEL_NO_FALLBACK))
    return set_error(OZK_ERR_RESIDUAL, "residual check failed at the selected S and fallback is disabled");
  return OZK_OK;
}

// --------------------------------------------------------------------- public API
extern "C" {

ozk_status_t ozk_create(ozk_handle_t* handle) {
  if (!handle) return set_error(OZK_ERR_ARG, "null handle pointer");
  ozk_context* h = new ozk_context();
  cudaGetDevice(&h->device);
  ozk_status_t st = cuda_check(cudaMalloc(&h->d_status, sizeof(int)), "cudaMalloc(status)");
  if (!st) st = cuda_check(cudaMemset(h->d_status, 0, sizeof(int)), "cudaMemset(status)");
  if (!st) {
    // the side stream at the lowest priority: its splits fill what the pivot-block inverses
    // on the handle's stream leave free
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    st = cuda_check(cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, least), "cudaStreamCreate(side)");
  }
  if (!st) st = cuda_check(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
  if (!st) st = cuda_check(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "cudaEventCreate");
  if (!st) st = cuda_check(cudaEventCreateWithFlags(&h->ev_join3, cudaEventDisableTiming), "cudaEventCreate");
  if (st) {
    if (h->d_status) cudaFree(h->d_status);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
    return st;
  }
  *handle = h;
  return OZK_OK;
}

ozk_status_t ozk_destroy(ozk_handle_t h) {
  if (!h) return OZK_OK;
  cudaStreamSynchronize(h->stream);
  if (h->aux) cudaStreamSynchronize(h->aux);
  if (h->ws) cudaFree(h->ws);
  if (h->d_status) cudaFree(h->d_status);
  if (h->sel_p) cudaFree(h->sel_p);
  if (h->sel_ws) cudaFree(h->sel_ws);
  if (h->sel_log_ws) cudaFree(h->sel_log_ws);
  if (h->one_ptrs) cudaFree(h->one_ptrs);
  if (h->sel_rec) cudaFree(h->sel_rec);
  for (auto& kv : h->tables) cudaFree(kv.second);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_join3) cudaEventDestroy(h->ev_join3);
  delete h;
  return OZK_OK;
}

ozk_status_t ozk_set_stream(ozk_handle_t h, void* stream) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  h->stream = static_cast<cudaStream_t>(stream);
  return OZK_OK;
}

ozk_status_t ozk_get_status(ozk_handle_t h, int* flags) {
  if (!h || !flags) return set_error(OZK_ERR_ARG, "null argument");
  ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  int v = 0;
  st = cuda_check(cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  if (st) return st;
  cudaMemset(h->d_status, 0, sizeof(int));
  *flags = v;
  return OZK_OK;
}

ozk_status_t ozk_reserve(ozk_handle_t h, size_t bytes) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  return ensure_ws(h, bytes);
}

size_t ozk_zgemm_workspace_size(int m, int n, int k, int S, int batch) {
  EmuGemm g;
  g.mmax = m; g.nmax = n; g.kmax = k; g.S = S; g.batch = batch;
  GemmPlan P;
  if (plan_gemm(g, &P)) return 0;
  return P.total;
}

const char* ozk_last_error(void) { return g_msg; }
uint64_t ozk_launch_count(void) { return g_launches; }

ozk_status_t ozaki_zgemm(ozk_handle_t h, char transa, char transb, int m, int n, int k, const double* alpha,
                         const void* A, int lda, const void* B, int ldb, const double* beta, void* C, int ldc,
                         int S, int pair_mode) {
  if (!h || !alpha || !beta) return set_error(OZK_ERR_ARG, "null argument");
  if (S < 0) return ozk_zgemm_dmma(h, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  EmuGemm g;
  if (!parse_op(transa, &g.oa) || !parse_op(transb, &g.ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  ozk_status_t st = check_dims(g.oa, g.ob, m, n, k, lda, ldb, ldc);
  if (st) return st;
  if (pair_mode != OZK_PAIRS_TRI && pair_mode != OZK_PAIRS_FULL) return set_error(OZK_ERR_ARG, "bad pair mode");
  if (m == 0 || n == 0) return OZK_OK;
  if (k == 0 || (alpha[0] == 0.0 && alpha[1] == 0.0)) {
    if (beta[0] == 1.0 && beta[1] == 0.0) return OZK_OK;
    launch_scale(m, n, static_cast<double2*>(C), ldc, beta[0], beta[1], h->stream);
    return cuda_check(cudaGetLastError(), "scale launch");
  }
  g.batch = 1; g.mmax = g.m = m; g.nmax = g.n = n; g.kmax = g.k = k;
  g.A = static_cast<const double2*>(A); g.lda = lda;
  g.B = static_cast<const double2*>(B); g.ldb = ldb;
  g.C = static_cast<double2*>(C); g.ldc = ldc;
  g.ar = alpha[0]; g.ai = alpha[1]; g.br = beta[0]; g.bi = beta[1];
  g.S = S; g.pair_mode = pair_mode;
  if (S == 0) return zgemm_auto(h, g);
  g.ksplit_ok = true;                         // the call owns the whole workspace
  return run_emulated(h, g);
}

// Ozaki-II tables for N moduli: the N largest pairwise-coprime integers <= 256 (greedy from 256
// down), powers of 256, Garner constants, and P (a product of at most 16 integers <= 256 fits
// in 128 bits).
static void oz2_tables(int N, Oz2Tables* T, unsigned __int128* Pout) {
  T->N = N;
  int cnt = 0;
  auto gcd = [](int a, int b) { while (b) { const int t = a % b; a = b; b = t; } return a; };
  for (int c = 256; c > 1 && cnt < N; --c) {
    bool ok = true;
    for (int j = 0; j < cnt; ++j) ok = ok && gcd(c, T->mod[j]) == 1;
    if (ok) T->mod[cnt++] = c;
  }
  unsigned __int128 P = 1;
  for (int t = 0; t < N; ++t) {
    const int m = T->mod[t];
    int pw = 1;
    for (int s = 0; s < 8; ++s) { T->pow256[t][s] = pw; pw = pw * 256 % m; }
    int prod = 1;                                      // m_0 ... m_{j-1} mod m_t
    for (int j = 0; j < t; ++j) { T->pm[t][j] = prod; prod = prod * T->mod[j] % m; }
    int inv = 1;                                        // prod^-1 mod m_t by search (m <= 256)
    for (int x = 1; x < m; ++x) if (prod * x % m == 1 % m) { inv = x; break; }
    T->inv[t] = t == 0 ? 1 : inv;
    P *= static_cast<unsigned>(m);
  }
  T->P_lo = static_cast<unsigned long long>(P);
  T->P_hi = static_cast<unsigned long long>(P >> 64);
  *Pout = P;
}

ozk_status_t ozaki2_zgemm(ozk_handle_t h, char transa, char transb, int m, int n, int k, const double* alpha,
                          const void* A, int lda, const void* B, int ldb, const double* beta, void* C, int ldc,
                          int nmod) {
  if (!h || !alpha || !beta) return set_error(OZK_ERR_ARG, "null argument");
  EmuGemm g;
  if (!parse_op(transa, &g.oa) || !parse_op(transb, &g.ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  ozk_status_t st = check_dims(g.oa, g.ob, m, n, k, lda, ldb, ldc);
  if (st) return st;
  if (nmod < 2 || nmod > OZ2_MAXMOD) return set_error(OZK_ERR_ARG, "number of moduli must be in 2..16");
  if (m == 0 || n == 0) return OZK_OK;
  if (k == 0 || (alpha[0] == 0.0 && alpha[1] == 0.0)) {
    if (beta[0] == 1.0 && beta[1] == 0.0) return OZK_OK;
    launch_scale(m, n, static_cast<double2*>(C), ldc, beta[0], beta[1], h->stream);
    return cuda_check(cudaGetLastError(), "scale launch");
  }
  if (k > 65536) return set_error(OZK_ERR_ARG, "Ozaki-II products are accumulated in int32: k <= 65536");
  Oz2Tables T{};
  unsigned __int128 P = 0;
  oz2_tables(nmod, &T, &P);
  // largest beta with 2k 4^beta < P / 2; |integer images| < 2^beta <= 2^63
  int bta = 0;
  int kbits = 0;
  for (unsigned long long v = 4ull * k; v; v >>= 1) ++kbits;
  while (bta < 63 && kbits + 2 * (bta + 1) <= 127) {
    const unsigned __int128 lhs = static_cast<unsigned __int128>(4ull * k) << (2 * (bta + 1));
    if (!(lhs < P)) break;
    ++bta;
  }
  if (bta < 1) return set_error(OZK_ERR_ARG, "too few moduli for this k");
  g.batch = 1; g.mmax = g.m = m; g.nmax = g.n = n; g.kmax = g.k = k;
  g.A = static_cast<const double2*>(A); g.lda = lda;
  g.B = static_cast<const double2*>(B); g.ldb = ldb;
  g.C = nullptr; g.ldc = m;
  g.S = nmod; g.pair_mode = PAIRS_DIAG; g.mode = EPI_RESIDUES;
  g.oz2 = &T; g.beta = bta;
  GemmPlan Pl;
  st = plan_gemm(g, &Pl);
  if (st) return st;
  const size_t rbytes = sizeof(int) * static_cast<size_t>(nmod) * m * 2 * n;
  const size_t off_r = align_up(Pl.total, 1024);
  st = ensure_ws(h, off_r + rbytes);
  if (st) return st;
  int* R = reinterpret_cast<int*>(static_cast<uint8_t*>(h->ws) + off_r);
  st = cuda_check(cudaMemsetAsync(R, 0, rbytes, h->stream), "clear products");
  if (st) return st;
  g.resid = R;
  g.ldres = 2LL * n;
  st = run_emulated(h, g);
  if (st) return st;
  CrtParams cp{};
  cp.R = R; cp.ldr = 2LL * n; cp.plane = static_cast<long long>(m) * 2 * n;
  cp.e = reinterpret_cast<const int*>(static_cast<uint8_t*>(h->ws) + Pl.offE);
  cp.f = reinterpret_cast<const int*>(static_cast<uint8_t*>(h->ws) + Pl.offF);
  cp.e_stride = Pl.rowsA; cp.f_stride = std::max(n, 1);
  cp.m = m; cp.n = n; cp.batch = 1; cp.beta = bta;
  cp.C = static_cast<double2*>(C); cp.ldc = ldc; cp.cstride = 0;
  cp.ar = alpha[0]; cp.ai = alpha[1]; cp.br = beta[0]; cp.bi = beta[1];
  cp.mode = (beta[0] == 0.0 && beta[1] == 0.0) ? EPI_STORE
            : ((alpha[0] == -1.0 && alpha[1] == 0.0 && beta[0] == 1.0 && beta[1] == 0.0) ? EPI_LU : EPI_GENERAL);
  {
    Prof pr(h, OZK_KIND_OTHER, 0.0, 8.0 * static_cast<double>(nmod) * m * 2 * n);
    launch_crt(cp, T, h->stream);
  }
  return cuda_check(cudaGetLastError(), "CRT launch");
}

ozk_status_t ozaki_zgemm_vbatched(ozk_handle_t h, char transa, char transb, const int* m, const int* n, const int* k,
                                  const double* alpha, const void* const* A, const int* lda, const void* const* B,
                                  const int* ldb, const double* beta, void* const* C, const int* ldc, int batch,
                                  int S, int pair_mode) {
  if (!h || !alpha || !beta || !m || !n || !k || !lda || !ldb || !ldc) return set_error(OZK_ERR_ARG, "null argument");
  if (batch < 0) return set_error(OZK_ERR_ARG, "negative batch");
  if (batch == 0) return OZK_OK;
  EmuGemm g;
  if (!parse_op(transa, &g.oa) || !parse_op(transb, &g.ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  if (pair_mode != OZK_PAIRS_TRI && pair_mode != OZK_PAIRS_FULL) return set_error(OZK_ERR_ARG, "bad pair mode");
  int mm = 0, nn = 0, kk = 0;
  for (int i = 0; i < batch; ++i) {
    ozk_status_t st = check_dims(g.oa, g.ob, m[i], n[i], k[i], lda[i], ldb[i], ldc[i]);
    if (st) return st;
    if (k[i] == 0) return set_error(OZK_ERR_ARG, "vbatched: k == 0 entries are not supported");
    mm = std::max(mm, m[i]); nn = std::max(nn, n[i]); kk = std::max(kk, k[i]);
  }
  if (mm == 0 || nn == 0) return OZK_OK;
  if (S == 0) return set_error(OZK_ERR_ARG, "vbatched: S = 0 (the selector) is a single-GEMM mode");
  g.batch = batch; g.mmax = mm; g.nmax = nn; g.kmax = kk;
  g.ar = alpha[0]; g.ai = alpha[1]; g.br = beta[0]; g.bi = beta[1];
  g.S = S; g.pair_mode = pair_mode;
  GemmPlan P;
  ozk_status_t st = OZK_OK;
  if (S > 0) {
    st = plan_gemm(g, &P);
    if (st) return st;
    st = ensure_ws(h, P.total);
    if (st) return st;
  }
  // device table of sizes: m, n, k, lda, ldb, ldc
  std::vector<int> tab(6 * static_cast<size_t>(batch));
  for (int i = 0; i < batch; ++i) {
    tab[i] = m[i]; tab[batch + i] = n[i]; tab[2 * batch + i] = k[i];
    tab[3 * batch + i] = lda[i]; tab[4 * batch + i] = ldb[i]; tab[5 * batch + i] = ldc[i];
  }
  const int* dtab = nullptr;
  st = size_table(h, std::move(tab), &dtab);
  if (st) return st;
  g.tm = dtab; g.tn = dtab + batch; g.tk = dtab + 2 * batch;
  g.tlda = dtab + 3 * batch; g.tldb = dtab + 4 * batch; g.tldc = dtab + 5 * batch;
  g.tA = reinterpret_cast<const double2* const*>(A);
  g.tB = reinterpret_cast<const double2* const*>(B);
  g.tC = reinterpret_cast<double2* const*>(C);
  g.sum_mnk = 0;
  for (int i = 0; i < batch; ++i) {
    g.sum_mnk += static_cast<double>(m[i]) * n[i] * k[i];
    g.sum_mk += static_cast<double>(m[i]) * k[i];
    g.sum_nk += static_cast<double>(n[i]) * k[i];
  }
  if (S < 0) {
    // binary64 DMMA GEMMs over the same tables (the native-precision baseline)
    DmmaParams d{};
    d.batch = batch; d.m = mm; d.n = nn; d.k = kk;
    d.transa = g.oa.trans; d.conja = g.oa.conj; d.transb = g.ob.trans; d.conjb = g.ob.conj;
    d.tm = g.tm; d.tn = g.tn; d.tk = g.tk;
    d.tA = g.tA; d.tlda = g.tlda; d.tB = g.tB; d.tldb = g.tldb; d.tC = g.tC; d.tldc = g.tldc;
    d.ar = g.ar; d.ai = g.ai; d.br = g.br; d.bi = g.bi;
    {
      Prof pr(h, OZK_KIND_DMMA, 8.0 * g.sum_mnk, 0.0);
      launch_dmma(d, h->stream);
    }
    return cuda_check(cudaGetLastError(), "batched DMMA launch");
  }
  return run_emulated(h, g);
}

ozk_status_t ozk_zgemm_dmma(ozk_handle_t h, char transa, char transb, int m, int n, int k, const double* alpha,
                            const void* A, int lda, const void* B, int ldb, const double* beta, void* C, int ldc) {
  if (!h || !alpha || !beta) return set_error(OZK_ERR_ARG, "null argument");
  OpFlags oa, ob;
  if (!parse_op(transa, &oa) || !parse_op(transb, &ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  ozk_status_t st = check_dims(oa, ob, m, n, k, lda, ldb, ldc);
  if (st) return st;
  if (m == 0 || n == 0) return OZK_OK;
  DmmaParams p{};
  p.m = m; p.n = n; p.k = k;
  p.transa = oa.trans; p.conja = oa.conj; p.transb = ob.trans; p.conjb = ob.conj;
  p.A = static_cast<const double2*>(A); p.lda = lda;
  p.B = static_cast<const double2*>(B); p.ldb = ldb;
  p.C = static_cast<double2*>(C); p.ldc = ldc;
  p.ar = alpha[0]; p.ai = alpha[1]; p.br = beta[0]; p.bi = beta[1];
  {
    Prof pr(h, OZK_KIND_DMMA, 8.0 * m * static_cast<double>(n) * k, 0.0);
    launch_dmma(p, h->stream);
  }
  return cuda_check(cudaGetLastError(), "DMMA launch");
}

ozk_status_t ozk_split_debug(ozk_handle_t h, int side, char trans, int rows, int k, const void* X, int ldx, int S,
                             int32_t* exps, int16_t* digits) {
  if (!h || !X || !exps) return set_error(OZK_ERR_ARG, "null argument");
  if (side != 0 && side != 1) return set_error(OZK_ERR_ARG, "side must be 0 or 1");
  if (rows <= 0 || k <= 0 || S < 1 || S > 16) return set_error(OZK_ERR_ARG, "bad size");
  OpFlags op;
  if (!parse_op(trans, &op)) return set_error(OZK_ERR_ARG, "bad trans flag");
  const int rows_out = side == 0 ? rows : 2 * rows;
  const int kpad = static_cast<int>(align_up(static_cast<size_t>(2 * k), 8));
  const size_t bytes = static_cast<size_t>(S) * rows_out * kpad * 2;
  ozk_status_t st = ensure_ws(h, bytes);
  if (st) return st;
  SplitParams sp{};
  sp.S = S; sp.nbits = 8 * S - 1; sp.status = h->d_status; sp.kpad = kpad; sp.side = side;
  sp.conj = op.conj;
  // side 0: op(X) is rows x k; side 1: op(X) is k x rows and its columns are the logical rows
  sp.trans = side == 0 ? op.trans : (op.trans ? 0 : 1);
  sp.out_rows = rows_out; sp.out = static_cast<__half*>(h->ws); sp.exps = exps; sp.exp_stride = rows;
  sp.X = nullptr; sp.X1 = static_cast<const double2*>(X); sp.ld1 = ldx; sp.rows1 = rows; sp.k1 = k;
  // debug digits are always dumped in the stacked layout [S][rows_out][2k]
  sp.dbg_digits = digits;
  launch_split(sp, rows, nullptr, 0, k, 1, h->stream);
  return cuda_check(cudaGetLastError(), "split launch");
}

ozk_status_t ozk_group_sums_debug(ozk_handle_t h, char transa, char transb, int m, int n, int k, const void* A,
                                  int lda, const void* B, int ldb, int S, int pair_mode, int64_t* groups) {
  if (!h || !groups) return set_error(OZK_ERR_ARG, "null argument");
  EmuGemm g;
  if (!parse_op(transa, &g.oa) || !parse_op(transb, &g.ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  ozk_status_t st = check_dims(g.oa, g.ob, m, n, k, lda, ldb, std::max(1, m));
  if (st) return st;
  if (m == 0 || n == 0 || k == 0) return set_error(OZK_ERR_ARG, "empty problem");
  g.batch = 1; g.mmax = g.m = m; g.nmax = g.n = n; g.kmax = g.k = k;
  g.A = static_cast<const double2*>(A); g.lda = lda;
  g.B = static_cast<const double2*>(B); g.ldb = ldb;
  g.C = nullptr; g.ldc = std::max(1, m);
  g.S = S; g.pair_mode = pair_mode; g.mode = 3;
  g.groups = reinterpret_cast<long long*>(groups);
  const int G = pair_mode == OZK_PAIRS_FULL ? 2 * S - 1 : S;
  st = cuda_check(cudaMemsetAsync(groups, 0, sizeof(int64_t) * static_cast<size_t>(G) * m * 2 * n, h->stream),
                  "memset groups");
  if (st) return st;
  return run_emulated(h, g);
}

ozk_status_t kkr_build_m(ozk_handle_t h, int L, int b, const void* t, const void* G, void* M) {
  if (!h || !t || !G || !M) return set_error(OZK_ERR_ARG, "null argument");
  if (L <= 0 || b <= 0) return set_error(OZK_ERR_ARG, "bad size");
  {
    const double nn = static_cast<double>(L) * b;
    Prof pr(h, OZK_KIND_BUILD_M, 8.0 * nn * nn * b, 32.0 * nn * nn);
    launch_build_m(L * b, b, static_cast<const double2*>(t), static_cast<const double2*>(G), static_cast<double2*>(M),
                   h->stream);
  }
  return cuda_check(cudaGetLastError(), "build_m launch");
}

static std::vector<int> tune_key(int nsolves, const int* n, int b, int S);

static ozk_status_t tau00_single(ozk_context* h, int n, int b, double2* M, const void* t0, void* tau, int S, int nb,
                                 size_t off_gemm, SelDefer* defer, int force_S);
static ozk_status_t tau00_batched_impl(ozk_handle_t h, int nsolves, const int* n, int b, void* const* M,
                                       const void* const* t0, void* const* tau, int S, int W, int w);

// tau_00 of one matrix: eliminate panels J = [p, q) from the trailing end, centre last.  Each
// panel: D^-1 of its pivot block (binary64 Gauss-Jordan), L = M_RJ D^-1 and M_RR -= L M_JR as
// emulated GEMMs with S slices (S >= 1), with the slice count the selector picks for each GEMM
// and its residual check (S = 0), or as binary64 DMMA GEMMs (S < 0).  With S = 0 the checks are
// recorded on the device and read once at the end: if any failed, M is restored from a copy
// taken at the start and the solve is redone with every GEMM at S = 10 (still checked).
ozk_status_t kkr_tau00(ozk_handle_t h, int n, int b, void* Mv, const void* t0, void* tau, int S, int nb) {
  if (!h || !Mv || !t0 || !tau) return set_error(OZK_ERR_ARG, "null argument");
  if (S > 16) return set_error(OZK_ERR_ARG, "S must be <= 16");
  const bool dmma = S < 0, auto_S = S == 0;
  if (auto_S) {
    if (!h->sel_ready)
      return set_error(OZK_ERR_ARG, "S = 0 needs selector parameters (ozk_selector_init, _load or _set_params)");
    if (capturing(h->stream))
      return set_error(OZK_ERR_CAPTURE, "S = 0 synchronises to read the selector's choices and cannot be captured");
  }
  if (nb == 0 && S >= 1 && b > 0 && b <= 64 && n > 0 && n % b == 0) {
    // emulated with a fixed S: the panel and leaf widths kkr_tau00_autotune_panels picks for one
    // matrix of this order (tuned on the first such call, cached); leaf panels run on the
    // batched solver (a single matrix's pivot inverses run on one SM each, so narrow leaves
    // inside wide panels cut the binary64 work that bounds the solve), whole panels below
    int W = 0, w = 0;
    auto it = h->tuned_nb.find(tune_key(1, &n, b, S));
    if (it != h->tuned_nb.end()) {
      W = it->second.first;
      w = it->second.second;
    } else {
      ozk_status_t st = kkr_tau00_autotune_panels(h, 1, &n, b, S, &W, &w, nullptr, nullptr, 0, nullptr);
      if (st) return st;
    }
    if (W == w) {
      nb = W;                     // whole panels: the single-matrix path has fewer launches per panel
    } else {
      if (!h->one_ptrs) {
        ozk_status_t st = cuda_check(cudaMalloc(&h->one_ptrs, 3 * sizeof(void*)), "cudaMalloc(pointer table)");
        if (st) { h->one_ptrs = nullptr; return st; }
      }
      launch_set_ptrs(h->one_ptrs, Mv, const_cast<void*>(t0), tau, h->stream);
      ozk_status_t st = cuda_check(cudaGetLastError(), "pointer table launch");
      if (st) return st;
      const int nn = n;
      return tau00_batched_impl(h, 1, &nn, b, h->one_ptrs, h->one_ptrs + 1, h->one_ptrs + 2, S, W, w);
    }
  }
  if (nb == 0 && b > 0 && b <= 64 && n > 0 && n % b == 0) {
    // the panel width kkr_tau00_autotune picks for one matrix of this size (S = 0: tuned at
    // S = 7), or 32 (binary64 DMMA)
    if (dmma) {
      nb = std::min(GJINV_MAX, (32 + b - 1) / b * b);
    } else {
      const int St = auto_S ? 7 : S;
      auto it = h->tuned_nb.find(tune_key(1, &n, b, St));
      if (it != h->tuned_nb.end() && it->second.first == it->second.second) {
        nb = it->second.first;
      } else {
        ozk_status_t st = kkr_tau00_autotune(h, 1, &n, b, St, &nb, nullptr);
        if (st) return st;
      }
    }
  }
  if (b <= 0 || n <= 0 || n % b || nb < b || nb % b || b > 64 || nb > GJINV_MAX)
    return set_error(OZK_ERR_ARG, "need n % b == 0, b <= 64, b <= nb <= 112, nb % b == 0");
  double2* M = static_cast<double2*>(Mv);
  // workspace: [D^-1, nb x nb][L scratch, n x nb (DMMA and S = 0)][S = 0: check record, copy
  // of M][GEMM workspace (emulated)]
  const size_t dinv_bytes = align_up(sizeof(double2) * nb * nb, 1024);
  const size_t ltmp_bytes = (dmma || auto_S) ? align_up(sizeof(double2) * static_cast<size_t>(n) * nb, 1024) : 0;
  const size_t mat_bytes = sizeof(double2) * static_cast<size_t>(n) * n;
  const size_t rec_bytes = auto_S ? 1024 : 0;
  const bool keep_copy = auto_S && !(h->sel_flags & OZK_SEL_NO_FALLBACK);
  const size_t copy_bytes = keep_copy ? align_up(mat_bytes, 1024) : 0;
  const size_t off_gemm = dinv_bytes + ltmp_bytes + rec_bytes + copy_bytes;
  {
    size_t need = off_gemm;
    if (!dmma) {
      EmuGemm probe;
      // S = 0: room for the fallback products (and for the reference products of a selector log)
      probe.mmax = n; probe.nmax = n; probe.kmax = nb; probe.S = auto_S ? (h->sel_log_f ? SEL_SREF : SEL_SMAX) : S;
      GemmPlan P;
      ozk_status_t st = plan_gemm(probe, &P);
      if (st) return st;
      need += P.total;
    }
    ozk_status_t st = ensure_ws(h, need);
    if (st) return st;
  }
  if (!auto_S) return tau00_single(h, n, b, M, t0, tau, S, nb, off_gemm, nullptr, 0);
  uint8_t* base = static_cast<uint8_t*>(h->ws);
  SelDefer* rec = reinterpret_cast<SelDefer*>(base + dinv_bytes + ltmp_bytes);
  double2* Mcopy = reinterpret_cast<double2*>(base + dinv_bytes + ltmp_bytes + rec_bytes);
  auto run_checked = [&](int force_S, SelDefer* out) -> ozk_status_t {
    ozk_status_t e = cuda_check(cudaMemsetAsync(rec, 0, sizeof(SelDefer), h->stream), "clear check record");
    if (!e) e = tau00_single(h, n, b, M, t0, tau, 0, nb, off_gemm, rec, force_S);
    if (!e) e = cuda_check(cudaMemcpyAsync(out, rec, sizeof(SelDefer), cudaMemcpyDeviceToHost, h->stream),
                           "read check record");
    if (!e) e = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return e;
  };
  ozk_status_t st = OZK_OK;
  if (keep_copy) st = cuda_check(cudaMemcpyAsync(Mcopy, M, mat_bytes, cudaMemcpyDeviceToDevice, h->stream), "copy M");
  SelDefer r1{};
  if (!st) st = run_checked(0, &r1);
  if (st) return st;
  ozk_selector_info info{};
  for (int o = 0; o < SEL_NO; ++o) {
    info.S_count[o] = r1.count[o];
    info.gemms += r1.count[o];
    if (r1.count[o]) info.S_selected = SEL_SMIN + o;
    info.predicted_log10_err[o] = r1.pred[o];
  }
  info.S_used = info.S_selected;
  info.residual = info.residual_selected = r1.max_resid;
  info.residual_ok = r1.failed ? 0 : 1;
  info.probe_seed = h->sel_seed + h->sel_calls - 1;
  if (r1.failed && keep_copy) {
    SelDefer r2{};
    st = cuda_check(cudaMemcpyAsync(M, Mcopy, mat_bytes, cudaMemcpyDeviceToDevice, h->stream), "restore M");
    if (!st) st = run_checked(SEL_SMAX, &r2);
    if (st) return st;
    info.S_used = SEL_SMAX;
    info.fallback = 1;
    info.residual = r2.max_resid;
    info.residual_ok = r2.failed ? 0 : 1;
  }
  h->sel_last = info;
  if (r1.failed && !keep_copy)
    return set_error(OZK_ERR_RESIDUAL, "a residual check of the solve failed and fallback is disabled");
  return OZK_OK;
}

static ozk_status_t tau00_single(ozk_context* h, int n, int b, double2* M, const void* t0, void* tau, int S, int nb,
                                 size_t off_gemm, SelDefer* defer, int force_S) {
  const bool dmma = S < 0, auto_S = S == 0;
  const size_t dinv_bytes = align_up(sizeof(double2) * nb * nb, 1024);
  double2* Dinv = static_cast<double2*>(h->ws);
  double2* Ltmp = reinterpret_cast<double2*>(static_cast<uint8_t*>(h->ws) + dinv_bytes);
  for (int q = n; q > b;) {
    const int p = std::max(q - nb, b), w = q - p, r = p;
    GjParams gj{};
    gj.D = nullptr; gj.D1 = M + p + static_cast<long long>(p) * n; gj.ldd1 = n; gj.nb1 = w;
    gj.X1 = Dinv; gj.ldx1 = w; gj.status = h->d_status;
    {
      Prof pr(h, OZK_KIND_GJ, 8.0 * w * w * w, 32.0 * w * w);
      launch_gjinv(gj, w, 1, h->stream);
    }
    double2* Lp = M + static_cast<long long>(p) * n;            // M[0:p, p:q]
    const double2* Up = M + p;                                   // M[p:q, 0:p]
    if (!dmma) {
      EmuGemm g1;                                                 // L = M_RJ D^-1
      g1.oa = {0, 0}; g1.ob = {0, 0}; g1.batch = 1;
      g1.mmax = g1.m = r; g1.nmax = g1.n = w; g1.kmax = g1.k = w;
      g1.A = Lp; g1.lda = n; g1.B = Dinv; g1.ldb = w;
      g1.S = S; g1.ar = 1; g1.br = 0;
      EmuGemm g2;                                                 // M_RR -= L M_JR
      g2.oa = {0, 0}; g2.ob = {0, 0}; g2.batch = 1;
      g2.mmax = g2.m = r; g2.nmax = g2.n = r; g2.kmax = g2.k = w;
      g2.A = Lp; g2.lda = n; g2.B = Up; g2.ldb = n; g2.C = M; g2.ldc = n;
      g2.S = S; g2.ar = -1; g2.br = 1;
      ozk_status_t st;
      if (!auto_S) {
        g1.C = Lp; g1.ldc = n;                                    // in place: both operands split first
        st = run_emulated(h, g1, off_gemm);
        if (!st) st = run_emulated(h, g2, off_gemm);
      } else {
        // the selector may recompute a product at S = 10, so L goes to the scratch (its operand
        // M_RJ stays intact) and is copied over M_RJ afterwards
        g1.C = Ltmp; g1.ldc = r;
        st = zgemm_auto(h, g1, off_gemm, defer, force_S);
        if (!st)
          st = cuda_check(cudaMemcpy2DAsync(Lp, sizeof(double2) * n, Ltmp, sizeof(double2) * r, sizeof(double2) * r,
                                            w, cudaMemcpyDeviceToDevice, h->stream),
                          "copy L panel");
        if (!st) st = zgemm_auto(h, g2, off_gemm, defer, force_S);
      }
      if (st) return st;
    } else {
      // binary64 DMMA baseline: L = M_RJ Dinv into the scratch, copy back, then update
      DmmaParams d1{};
      d1.m = r; d1.n = w; d1.k = w; d1.A = Lp; d1.lda = n; d1.B = Dinv; d1.ldb = w;
      d1.C = Ltmp; d1.ldc = r; d1.ar = 1; d1.br = 0;
      {
        Prof pr(h, OZK_KIND_DMMA, 8.0 * r * static_cast<double>(w) * w, 0.0);
        launch_dmma(d1, h->stream);
      }
      ozk_status_t st = cuda_check(cudaMemcpy2DAsync(Lp, sizeof(double2) * n, Ltmp, sizeof(double2) * r,
                                                     sizeof(double2) * r, w, cudaMemcpyDeviceToDevice, h->stream),
                                   "copy L panel");
      if (st) return st;
      DmmaParams d2{};
      d2.m = r; d2.n = r; d2.k = w; d2.A = Lp; d2.lda = n; d2.B = Up; d2.ldb = n; d2.C = M; d2.ldc = n;
      d2.ar = -1; d2.br = 1;
      {
        Prof pr(h, OZK_KIND_DMMA, 8.0 * r * static_cast<double>(r) * w, 0.0);
        launch_dmma(d2, h->stream);
      }
    }
    q = p;
  }
  GjParams gj{};
  gj.D = nullptr; gj.D1 = M; gj.ldd1 = n; gj.nb1 = b;
  gj.R1 = static_cast<const double2*>(t0); gj.ldr1 = b; gj.nrhs = b;
  gj.X1 = static_cast<double2*>(tau); gj.ldx1 = b; gj.status = h->d_status;
  {
    Prof pr(h, OZK_KIND_GJ, 8.0 * b * b * 2.0 * b, 48.0 * b * b);
    launch_gj(gj, b, b, 1, h->stream);
  }
  return cuda_check(cudaGetLastError(), "kkr_tau00 launches");
}

// ---- emulated ZTRSM (right side) and the LU-based tau_00
// X T = B solved in place (B := X), B m x w, T w x w triangular, by block columns of ZTRSM_BT:
// block column j of X is (B_j - the solved columns times T's block column j) times the inverse
// of T's diagonal block; the update and the product by the block inverse are emulated GEMMs,
// the block inverse is binary64.  Upper T: block columns in order 0, 1, ...; lower: from the
// last.  Workspace at ws_offset: the block inverse, then the GEMM workspace.
constexpr int ZTRSM_BT = 16;

static ozk_status_t ztrsm_right(ozk_context* h, bool upper, bool unit, int m, int w, const double2* T, long long ldt,
                                double2* B, long long ldb, int S, size_t ws_offset) {
  const int bt = ZTRSM_BT;
  const int nblk = (w + bt - 1) / bt;
  double2* tinv = reinterpret_cast<double2*>(static_cast<uint8_t*>(h->ws) + ws_offset);
  const size_t gemm_off = ws_offset + align_up(sizeof(double2) * bt * bt, 1024);
  for (int step = 0; step < nblk; ++step) {
    const int j = upper ? step : nblk - 1 - step;
    const int c0 = j * bt, r = std::min(bt, w - c0);
    double2* Bj = B + static_cast<long long>(c0) * ldb;
    const int k0 = upper ? 0 : c0 + r;             // first solved column used by the update
    const int kk = upper ? c0 : w - c0 - r;        // number of solved columns
    if (kk > 0 && m > 0) {
      EmuGemm g;                                   // B_j -= X_solved T[solved, block j]
      g.oa = {0, 0}; g.ob = {0, 0}; g.batch = 1;
      g.mmax = g.m = m; g.nmax = g.n = r; g.kmax = g.k = kk;
      g.A = B + static_cast<long long>(k0) * ldb; g.lda = static_cast<int>(ldb);
      g.B = T + k0 + static_cast<long long>(c0) * ldt; g.ldb = static_cast<int>(ldt);
      g.C = Bj; g.ldc = static_cast<int>(ldb);
      g.S = S; g.ar = -1; g.br = 1;
      ozk_status_t st = run_emulated(h, g, gemm_off);
      if (st) return st;
    }
    {
      Prof pr(h, OZK_KIND_GJ, 8.0 * r * r * r / 3.0, 32.0 * r * r);
      launch_tri_inv(T + c0 + static_cast<long long>(c0) * ldt, ldt, r, upper ? 1 : 0, unit ? 1 : 0, tinv, bt,
                     h->d_status, h->stream);
    }
    if (m > 0) {
      EmuGemm g;                                   // B_j := B_j T_jj^-1 (in place: A is split first)
      g.oa = {0, 0}; g.ob = {0, 0}; g.batch = 1;
      g.mmax = g.m = m; g.nmax = g.n = r; g.kmax = g.k = r;
      g.A = Bj; g.lda = static_cast<int>(ldb); g.B = tinv; g.ldb = bt; g.C = Bj; g.ldc = static_cast<int>(ldb);
      g.S = S; g.ar = 1; g.br = 0;
      ozk_status_t st = run_emulated(h, g, gemm_off);
      if (st) return st;
    }
  }
  return OZK_OK;
}

static size_t ztrsm_ws_bytes(int m, int w, int S, ozk_status_t* st) {
  EmuGemm probe;
  probe.mmax = std::max(m, 1); probe.nmax = ZTRSM_BT; probe.kmax = std::max(w, ZTRSM_BT); probe.S = S;
  GemmPlan P;
  *st = plan_gemm(probe, &P);
  return align_up(sizeof(double2) * ZTRSM_BT * ZTRSM_BT, 1024) + P.total;
}

ozk_status_t ozaki_ztrsm(ozk_handle_t h, char uplo, char diag, int m, int n, const void* T, int ldt, void* B, int ldb,
                         int S) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  const bool upper = uplo == 'U' || uplo == 'u', unit = diag == 'U' || diag == 'u';
  if (!(upper || uplo == 'L' || uplo == 'l') || !(unit || diag == 'N' || diag == 'n'))
    return set_error(OZK_ERR_ARG, "uplo must be 'U' or 'L', diag 'N' or 'U'");
  if (m < 0 || n < 0) return set_error(OZK_ERR_ARG, "negative dimension");
  if (S < 1 || S > 16) return set_error(OZK_ERR_ARG, "S must be in 1..16");
  if (m == 0 || n == 0) return OZK_OK;
  if (!T || !B) return set_error(OZK_ERR_ARG, "null argument");
  if (ldt < n || ldb < m) return set_error(OZK_ERR_ARG, "ldt < n or ldb < m");
  ozk_status_t st = OZK_OK;
  const size_t need = ztrsm_ws_bytes(m, n, S, &st);
  if (st) return st;
  st = ensure_ws(h, need);
  if (st) return st;
  st = ztrsm_right(h, upper, unit, m, n, static_cast<const double2*>(T), ldt, static_cast<double2*>(B), ldb, S, 0);
  if (st) return st;
  return cuda_check(cudaGetLastError(), "ozaki_ztrsm launches");
}

// tau_00 with the pivot blocks factored instead of inverted: per panel P D = L U (binary64,
// partial pivoting, the interchanges also applied to the row strip M_JR), M_RJ := M_RJ U^-1 L^-1
// by two emulated right-side ZTRSMs, M_RR -= M_RJ (P M_JR) by an emulated GEMM -- the
// ZGEMM + ZTRSM mix of an LU-based inversion.  Same Schur complement S_00 as kkr_tau00.
ozk_status_t kkr_tau00_lu(ozk_handle_t h, int n, int b, void* Mv, const void* t0, void* tau, int S, int nb) {
  if (!h || !Mv || !t0 || !tau) return set_error(OZK_ERR_ARG, "null argument");
  if (S < 1) return set_error(OZK_ERR_ARG, "the LU variant runs emulated GEMMs (S >= 1)");
  if (b <= 0 || n <= 0 || n % b || nb < b || nb % b || b > 64 || nb > GJINV_MAX)
    return set_error(OZK_ERR_ARG, "need n % b == 0, b <= 64, b <= nb <= 112, nb % b == 0");
  double2* M = static_cast<double2*>(Mv);
  ozk_status_t st = OZK_OK;
  size_t need = ztrsm_ws_bytes(n, nb, S, &st);
  if (st) return st;
  {
    EmuGemm probe;
    probe.mmax = n; probe.nmax = n; probe.kmax = nb; probe.S = S;
    GemmPlan P;
    st = plan_gemm(probe, &P);
    if (st) return st;
    need = std::max(need, P.total);
  }
  st = ensure_ws(h, need);
  if (st) return st;
  for (int q = n; q > b;) {
    const int p = std::max(q - nb, b), w = q - p;
    double2* D = M + p + static_cast<long long>(p) * n;
    double2* Lp = M + static_cast<long long>(p) * n;            // M[0:p, p:q]
    double2* Up = M + p;                                         // M[p:q, 0:p]
    {
      Prof pr(h, OZK_KIND_GJ, 8.0 * w * w * w / 3.0, 32.0 * w * w);
      launch_lu_panel(D, n, w, Up, n, p, h->d_status, h->stream);
    }
    st = ztrsm_right(h, true, false, p, w, D, n, Lp, n, S, 0);    // M_RJ U^-1
    if (st) return st;
    st = ztrsm_right(h, false, true, p, w, D, n, Lp, n, S, 0);    // then L^-1 (unit lower)
    if (st) return st;
    EmuGemm g2;                                                   // M_RR -= M_RJ (P M_JR)
    g2.oa = {0, 0}; g2.ob = {0, 0}; g2.batch = 1;
    g2.mmax = g2.m = p; g2.nmax = g2.n = p; g2.kmax = g2.k = w;
    g2.A = Lp; g2.lda = n; g2.B = Up; g2.ldb = n; g2.C = M; g2.ldc = n;
    g2.S = S; g2.ar = -1; g2.br = 1;
    st = run_emulated(h, g2, 0);
    if (st) return st;
    q = p;
  }
  GjParams gj{};
  gj.D = nullptr; gj.D1 = M; gj.ldd1 = n; gj.nb1 = b;
  gj.R1 = static_cast<const double2*>(t0); gj.ldr1 = b; gj.nrhs = b;
  gj.X1 = static_cast<double2*>(tau); gj.ldx1 = b; gj.status = h->d_status;
  {
    Prof pr(h, OZK_KIND_GJ, 8.0 * b * b * 2.0 * b, 48.0 * b * b);
    launch_gj(gj, b, b, 1, h->stream);
  }
  return cuda_check(cudaGetLastError(), "kkr_tau00_lu launches");
}

// Shared-G build.  Lh (HOST, per atom) may be null: every atom has L sites and G has order L b;
// otherwise atom a has Lh[a] sites, L = max Lh[a], and its G is the leading block of G (ld ldg).
static ozk_status_t build_m_shared_impl(ozk_context* h, int natoms, const int* Lh, int L, int b,
                                        const void* const* t, const void* G, int ldg, void* const* M, int S) {
  const long long rows = static_cast<long long>(natoms) * b, n = static_cast<long long>(L) * b;
  if (rows > (1 << 30) || n > (1 << 30)) return set_error(OZK_ERR_ARG, "sizes too large");
  if (ldg < n) return set_error(OZK_ERR_ARG, "ldg smaller than the largest L b");
  // block row i of every atom's M: I - (t_{a,i} stacked over the atoms) G[ib:(i+1)b, :], one
  // emulated GEMM per i (m = natoms b, n = L b, k = b), the rows scattered back to the atoms
  const size_t stack_bytes = align_up(sizeof(double2) * static_cast<size_t>(L) * rows * b, 1024);
  const int* dL = nullptr;
  const int* dn = nullptr;
  double sum_n2 = static_cast<double>(natoms) * n * n;       // useful outputs: sum of n_a^2
  {
    ozk_status_t st = table_room(h, 8);
    if (st) return st;
  }
  if (Lh) {
    std::vector<int> nv(natoms);
    sum_n2 = 0;
    for (int a = 0; a < natoms; ++a) { nv[a] = Lh[a] * b; sum_n2 += static_cast<double>(nv[a]) * nv[a]; }
    ozk_status_t st = size_table(h, std::vector<int>(Lh, Lh + natoms), &dL);
    if (st) return st;
    st = size_table(h, std::move(nv), &dn);
    if (st) return st;
  }
  // mixed sizes: the atoms stacked by decreasing LIZ (ties in input order), and block row i
  // cut into problems of up to 128 stacked rows, each as wide as its first (largest) atom: the
  // stacked rows of atoms without block row i and the columns past an atom's order are never
  // enumerated as tiles (only their rows inside a partly used tile are, and are not written)
  const int* dperm = nullptr;
  const int* dremap = nullptr;
  const int* dgm = nullptr;
  const int* dgn = nullptr;
  int nprob = 0;
  if (Lh && natoms > 1) {
    std::vector<int> perm(natoms);
    for (int a = 0; a < natoms; ++a) perm[a] = a;
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return Lh[x] > Lh[y]; });
    std::vector<int> remap, gm, gn;
    for (int i = 0; i < L; ++i) {
      int cnt = 0;                                   // atoms with block row i: a prefix of the order
      while (cnt < natoms && Lh[perm[cnt]] > i) ++cnt;
      const long long live = static_cast<long long>(cnt) * b;
      for (long long r0 = 0; r0 < live; r0 += 128) {
        remap.push_back(i);
        remap.push_back(static_cast<int>(r0));
        gm.push_back(static_cast<int>(std::min<long long>(128, live - r0)));
        gn.push_back(Lh[perm[r0 / b]] * b);
      }
    }
    nprob = static_cast<int>(gm.size());
    ozk_status_t st = size_table(h, std::move(perm), &dperm);
    if (!st) st = size_table(h, std::move(remap), &dremap);
    if (!st) st = size_table(h, std::move(gm), &dgm);
    if (!st) st = size_table(h, std::move(gn), &dgn);
    if (st) return st;
  }
  EmuGemm g;
  g.oa = {0, 0}; g.ob = {0, 0}; g.batch = L;
  g.mmax = g.m = static_cast<int>(rows); g.nmax = g.n = static_cast<int>(n); g.kmax = g.k = b;
  if (dremap) {
    g.remap = dremap; g.gbatch = nprob; g.gm = dgm; g.gn = dgn;
    g.crow_perm = dperm;
  }
  g.lda = static_cast<int>(rows); g.zsA = rows * b;
  g.B = static_cast<const double2*>(G); g.ldb = ldg; g.zsB = b;
  g.C = nullptr; g.ldc = static_cast<int>(n);
  g.crow = reinterpret_cast<double2* const*>(M); g.crow_b = b; g.crow_n = dn;
  g.mode = EPI_IMINUS; g.S = S;
  g.sum_mnk = sum_n2 * b;
  g.sum_mk = static_cast<double>(L) * rows * b;
  g.sum_nk = static_cast<double>(L) * n * b;
  GemmPlan P;
  ozk_status_t st = plan_gemm(g, &P);
  if (st) return st;
  st = ensure_ws(h, stack_bytes + P.total);
  if (st) return st;
  double2* stack = static_cast<double2*>(h->ws);
  g.A = stack;
  {
    Prof pr(h, OZK_KIND_BUILD_M, 0.0, 32.0 * static_cast<double>(L) * rows * b);
    launch_stack_t(reinterpret_cast<const double2* const*>(t), dL, dperm, natoms, L, b, stack, h->stream);
  }
  st = cuda_check(cudaGetLastError(), "stack_t launch");
  if (st) return st;
  return run_emulated(h, g, stack_bytes);
}

ozk_status_t kkr_build_m_shared(ozk_handle_t h, int natoms, int L, int b, const void* const* t, const void* G,
                                void* const* M, int S) {
  if (!h || !t || !G || !M) return set_error(OZK_ERR_ARG, "null argument");
  if (natoms < 0 || L < 1 || b < 1) return set_error(OZK_ERR_ARG, "need natoms >= 0, L >= 1, b >= 1");
  if (S < 1 || S > 16) return set_error(OZK_ERR_ARG, "S must be in 1..16");
  if (natoms == 0) return OZK_OK;
  return build_m_shared_impl(h, natoms, nullptr, L, b, t, G, L * b, M, S);
}

ozk_status_t kkr_build_m_shared_sizes(ozk_handle_t h, int natoms, const int* L, int b, const void* const* t,
                                      const void* G, int ldg, void* const* M, int S) {
  if (!h || !L || !t || !G || !M) return set_error(OZK_ERR_ARG, "null argument");
  if (natoms < 0 || b < 1) return set_error(OZK_ERR_ARG, "need natoms >= 0, b >= 1");
  if (S < 1 || S > 16) return set_error(OZK_ERR_ARG, "S must be in 1..16");
  if (natoms == 0) return OZK_OK;
  int Lmax = 0;
  for (int a = 0; a < natoms; ++a) {
    if (L[a] < 1) return set_error(OZK_ERR_ARG, "every L[a] must be >= 1");
    Lmax = std::max(Lmax, L[a]);
  }
  return build_m_shared_impl(h, natoms, L, Lmax, b, t, G, ldg, M, S);
}

// Batched block LU of `nsolves` matrices in lockstep.  Panels J = [p, q) of width W are
// eliminated from the trailing end of every M, each leaf by leaf (leaves of width w from the
// panel's end, the front one narrower when w does not divide the panel): per leaf [a, hi) the
// pivot block's binary64 inverse, L = M[0:a, a:hi] D^-1 in place, and the leaf's update of the
// frame of [0, a) x [0, a) outside [0, p) x [0, p); per panel the deferred update
// M[0:p, 0:p] -= M[0:p, p:q] M[p:q, 0:p] with K = W (w = W: one leaf, no frame, the plain
// panel-by-panel block LU).
static ozk_status_t tau00_batched_impl(ozk_handle_t h, int nsolves, const int* n, int b, void* const* M,
                                       const void* const* t0, void* const* tau, int S, int W, int w) {
  if (!h || !n || !M || !t0 || !tau) return set_error(OZK_ERR_ARG, "null argument");
  if (nsolves < 0) return set_error(OZK_ERR_ARG, "negative nsolves");
  if (nsolves == 0) return OZK_OK;
  if (S == 0) return set_error(OZK_ERR_ARG, "S = 0 is resolved to a slice count before the solves");
  if (w == 0) w = W;
  const bool dmma = S < 0;                     // binary64 DMMA GEMMs instead of emulated ones
  if (b <= 0 || b > 64 || w < b || w % b || w > GJINV_MAX || W < w || W % b || W > OZK_PANEL_MAX)
    return set_error(OZK_ERR_ARG, "need b <= 64, b <= w <= 112, w <= W <= 448, w and W multiples of b");
  if (dmma && W != w) return set_error(OZK_ERR_ARG, "the binary64 DMMA solve eliminates whole panels (w = W)");
  const int nleaves = (W + w - 1) / w;
  int nmax = 0;
  for (int i = 0; i < nsolves; ++i) {
    if (n[i] <= 0 || n[i] % b) return set_error(OZK_ERR_ARG, "every n[i] must be a positive multiple of b");
    nmax = std::max(nmax, n[i]);
  }
  const int panels = (nmax - b + W - 1) / W;
  // workspace layout: [D^-1 per solve, w x w][step tables][GEMM 1 workspace][GEMM 2 workspace]
  // [GEMM 3 workspace] -- separate GEMM workspaces, so that the early operand splits of GEMMs 1
  // and 2 can run on the side stream while the pivot blocks are inverted
  const size_t ns = static_cast<size_t>(nsolves);
  const size_t off_dinv = 0;
  const size_t off_tab = align_up(off_dinv + ns * w * w * sizeof(double2), 1024);
  const size_t n_ptr = 11, n_int = 26;
  const size_t off_g1 = align_up(off_tab + ns * (n_ptr * sizeof(void*) + n_int * sizeof(int)), 1024);
  size_t off_g2 = off_g1, off_g3 = off_g1, total = off_g1;
  ozk_status_t st = OZK_OK;
  if (!dmma) {
    EmuGemm probe;
    probe.batch = nsolves; probe.mmax = nmax; probe.nmax = w; probe.kmax = w; probe.S = S;
    GemmPlan P;
    st = plan_gemm(probe, &P);
    if (st) return st;
    off_g2 = align_up(off_g1 + P.total, 1024);
    probe.nmax = nmax;
    st = plan_gemm(probe, &P);
    if (st) return st;
    off_g3 = align_up(off_g2 + P.total, 1024);
    probe.kmax = W;
    st = plan_gemm(probe, &P);
    if (st) return st;
    total = off_g3 + P.total;
  } else {
    // binary64 path: L = M_RJ D^-1 of every solve into its own nmax x w scratch (a tiled GEMM
    // cannot overwrite its own operand), then pointer and leading-dimension tables of it
    total = align_up(off_g1 + ns * nmax * w * sizeof(double2), 1024) + ns * (sizeof(void*) + sizeof(int));
  }
  st = ensure_ws(h, total);
  if (st) return st;
  const int* dn = nullptr;
  st = size_table(h, std::vector<int>(n, n + nsolves), &dn);
  if (st) return st;
  uint8_t* ws = static_cast<uint8_t*>(h->ws);
  double2* dinv = reinterpret_cast<double2*>(ws + off_dinv);
  uint8_t* pp = ws + off_tab;                  // ns x n_ptr pointer slots
  int* pi = reinterpret_cast<int*>(ws + off_tab + ns * n_ptr * sizeof(void*));
  auto slot = [&](int k) { return pp + k * ns * sizeof(void*); };
  KkrStep t;
  t.D = reinterpret_cast<const double2**>(slot(0)); t.X = reinterpret_cast<double2**>(slot(1));
  t.A1 = reinterpret_cast<const double2**>(slot(2)); t.B1 = reinterpret_cast<const double2**>(slot(3));
  t.C1 = reinterpret_cast<double2**>(slot(4)); t.A2 = reinterpret_cast<const double2**>(slot(5));
  t.B2 = reinterpret_cast<const double2**>(slot(6)); t.C2 = reinterpret_cast<double2**>(slot(7));
  t.A3 = reinterpret_cast<const double2**>(slot(8)); t.B3 = reinterpret_cast<const double2**>(slot(9));
  t.C3 = reinterpret_cast<double2**>(slot(10));
  int k = 0;
  auto ints = [&]() { return pi + (k++) * ns; };
  t.ldd = ints(); t.nbv = ints(); t.ldx = ints();
  t.lda1 = ints(); t.ldb1 = ints(); t.ldc1 = ints(); t.m1 = ints(); t.n1 = ints(); t.k1 = ints();
  t.lda2 = ints(); t.ldb2 = ints(); t.ldc2 = ints(); t.m2 = ints(); t.n2 = ints(); t.k2 = ints();
  t.skm2 = ints(); t.skn2 = ints();
  t.lda3 = ints(); t.ldb3 = ints(); t.ldc3 = ints(); t.m3 = ints(); t.n3 = ints(); t.k3 = ints();
  if (static_cast<size_t>(k) > n_int) return set_error(OZK_ERR_ARG, "step table layout");
  double2* const* Mp = reinterpret_cast<double2* const*>(M);
  double2** tL = nullptr;
  int* tLld = nullptr;
  if (dmma) {
    const size_t off_lt = align_up(off_g1 + ns * nmax * w * sizeof(double2), 1024);
    tL = reinterpret_cast<double2**>(ws + off_lt);
    tLld = reinterpret_cast<int*>(ws + off_lt + ns * sizeof(void*));
    launch_strided_ptrs(tL, tLld, reinterpret_cast<double2*>(ws + off_g1), static_cast<long long>(nmax) * w, nmax,
                        nsolves, h->stream);
  }

  auto gemm_tables = [&](int which, int mmax, int nmaxg, int kmax, double smnk, double smk, double snk, bool lu,
                         int sides, bool gemm, cudaStream_t stream, int box) -> ozk_status_t {
    EmuGemm g;
    g.oa = {0, 0}; g.ob = {0, 0}; g.batch = nsolves; g.mmax = mmax; g.nmax = nmaxg; g.kmax = kmax; g.S = S;
    if (which == 1) {
      g.tA = t.A1; g.tlda = t.lda1; g.tB = t.B1; g.tldb = t.ldb1; g.tC = t.C1; g.tldc = t.ldc1;
      g.tm = t.m1; g.tn = t.n1; g.tk = t.k1;
    } else if (which == 2) {
      g.tA = t.A2; g.tlda = t.lda2; g.tB = t.B2; g.tldb = t.ldb2; g.tC = t.C2; g.tldc = t.ldc2;
      g.tm = t.m2; g.tn = t.n2; g.tk = t.k2;
      g.tskm = t.skm2; g.tskn = t.skn2; g.box_m = box; g.box_n = box;
    } else {
      g.tA = t.A3; g.tlda = t.lda3; g.tB = t.B3; g.tldb = t.ldb3; g.tC = t.C3; g.tldc = t.ldc3;
      g.tm = t.m3; g.tn = t.n3; g.tk = t.k3;
    }
    g.ar = lu ? -1 : 1; g.br = lu ? 1 : 0;
    g.sum_mnk = smnk; g.sum_mk = smk; g.sum_nk = snk;
    g.split_sides = sides; g.run_gemm = gemm; g.stream = stream;
    return run_emulated(h, g, which == 1 ? off_g1 : (which == 2 ? off_g2 : off_g3));
  };

  // leaf j of panel s: every solve's sizes (host mirror of kkr_step_kernel) for the launch
  // extents and the profiler's algorithmic counts
  for (int s = 0; s < panels; ++s) {
    for (int j = 0; j < nleaves; ++j) {
      int amax = 0, wmax = 0, fmax = 0, pmax3 = 0, kmax3 = 0, nact = 0, box = 0;
      double s1 = 0, sa1 = 0, sw1 = 0, sw3g = 0, sw2 = 0, s2 = 0, sa2 = 0, sb2 = 0, s3 = 0, sa3 = 0;
      bool any3 = false, any2 = false;
      for (int i = 0; i < nsolves; ++i) {
        const int q = n[i] - s * W;
        if (q <= b) continue;
        const int p = std::max(q - W, b);
        if (j == nleaves - 1) {
          any3 = true;
          pmax3 = std::max(pmax3, p);
          kmax3 = std::max(kmax3, q - p);
          s3 += static_cast<double>(p) * p * (q - p);
          sa3 += static_cast<double>(p) * (q - p);
        }
        const int hi = q - j * w;
        if (hi <= p) continue;
        const int a = std::max(hi - w, p), wl = hi - a;
        ++nact;
        amax = std::max(amax, a);
        wmax = std::max(wmax, wl);
        s1 += static_cast<double>(a) * wl * wl;
        sa1 += static_cast<double>(a) * wl;
        sw1 += static_cast<double>(wl) * wl;
        sw3g += static_cast<double>(wl) * wl * wl;
        if (a > p) {
          // the frame: rows [p, a) x [0, a) and rows [0, p) x [p, a)
          any2 = true;
          fmax = std::max(fmax, a);
          box = box == 0 ? p : std::min(box, p);
          const double fr = static_cast<double>(a) * a - static_cast<double>(p) * p;
          s2 += fr * wl;
          sa2 += static_cast<double>(a) * wl;
          sb2 += static_cast<double>(a) * wl;
          sw2 += fr;
        }
      }
      if (nact == 0 && !any3) continue;
      bool early3 = false;                           // GEMM 3's right operand split on the side stream
      {
        Prof pr(h, OZK_KIND_OTHER, 0.0, 0.0);
        launch_kkr_step(s, j, nleaves, nsolves, dn, Mp, b, W, w, dinv, t, h->stream);
      }
      if (dmma) {
        // one leaf per panel (w = W): the GEMM 3 of this leaf is the trailing update
        GjParams gj{};
        gj.D = t.D; gj.ldd = t.ldd; gj.nb = t.nbv; gj.R = nullptr; gj.X = t.X; gj.ldx = t.ldx; gj.nrhs = 0;
        gj.status = h->d_status;
        {
          Prof pr(h, OZK_KIND_GJ, 8.0 * sw3g, 32.0 * sw1);
          launch_gjinv(gj, wmax, nsolves, h->stream);
        }
        DmmaParams d1{};                                   // L = M_RJ D^-1 into the scratch
        d1.batch = nsolves; d1.m = amax; d1.n = wmax; d1.k = wmax;
        d1.tm = t.m1; d1.tn = t.n1; d1.tk = t.k1;
        d1.tA = t.A1; d1.tlda = t.lda1; d1.tB = t.B1; d1.tldb = t.ldb1; d1.tC = tL; d1.tldc = tLld;
        d1.ar = 1; d1.br = 0;
        {
          Prof pr(h, OZK_KIND_DMMA, 8.0 * s1, 0.0);
          launch_dmma(d1, h->stream);
        }
        DmmaParams d2{};                                   // M_RR -= L M_JR
        d2.batch = nsolves; d2.m = pmax3; d2.n = pmax3; d2.k = kmax3;
        d2.tm = t.m3; d2.tn = t.n3; d2.tk = t.k3;
        d2.tA = tL; d2.tlda = tLld; d2.tB = t.B3; d2.tldb = t.ldb3; d2.tC = t.C3; d2.tldc = t.ldc3;
        d2.ar = -1; d2.br = 1;
        {
          Prof pr(h, OZK_KIND_DMMA, 8.0 * s3, 0.0);
          launch_dmma(d2, h->stream);
        }
        continue;
      }
      if (nact > 0) {
        // M_RJ of the leaf (GEMM 1's A) and its U rows (GEMM 2's B) do not depend on D^-1: they
        // are split on the side stream while the pivot blocks are inverted
        st = cuda_check(cudaEventRecord(h->ev_fork, h->stream), "record fork");
        if (!st) st = cuda_check(cudaStreamWaitEvent(h->aux, h->ev_fork, 0), "side stream wait");
        if (st) return st;
        GjParams gj{};
        gj.D = t.D; gj.ldd = t.ldd; gj.nb = t.nbv; gj.R = nullptr; gj.X = t.X; gj.ldx = t.ldx; gj.nrhs = 0;
        gj.status = h->d_status;
        {
          Prof pr(h, OZK_KIND_GJ, 8.0 * sw3g, 32.0 * sw1);
          launch_gjinv(gj, wmax, nsolves, h->stream);
        }
        st = gemm_tables(1, amax, wmax, wmax, s1, sa1, sw1, false, 1, false, h->aux, 0);
        if (!st && any2) st = gemm_tables(2, fmax, fmax, wmax, s2, sa2, sb2, true, 2, false, h->aux, box);
        if (!st) st = cuda_check(cudaEventRecord(h->ev_join, h->aux), "record join");
        // last leaf: the U rows M[p:q, 0:p] of the deferred update are final (the earlier
        // leaves' frame updates were their last writers), so they are split on the side stream
        // too, joined only before the deferred update
        if (!st && any3) {
          early3 = true;
          st = gemm_tables(3, pmax3, pmax3, kmax3, s3, sa3, sa3, true, 2, false, h->aux, 0);
          if (!st) st = cuda_check(cudaEventRecord(h->ev_join3, h->aux), "record join");
        }
        if (!st) st = cuda_check(cudaStreamWaitEvent(h->stream, h->ev_join, 0), "join side stream");
        if (st) return st;
        st = gemm_tables(1, amax, wmax, wmax, s1, sa1, sw1, false, 2, true, h->stream, 0);
        if (st) return st;
        if (any2) {
          st = gemm_tables(2, fmax, fmax, wmax, s2, sa2, sb2, true, 1, true, h->stream, box);
          if (st) return st;
        }
      }
      if (any3) {
        if (early3) {
          st = cuda_check(cudaStreamWaitEvent(h->stream, h->ev_join3, 0), "join side stream");
          if (!st) st = gemm_tables(3, pmax3, pmax3, kmax3, s3, sa3, sa3, true, 1, true, h->stream, 0);
        } else {
          st = gemm_tables(3, pmax3, pmax3, kmax3, s3, sa3, sa3, true, 3, true, h->stream, 0);
        }
        if (st) return st;
      }
    }
  }
  {
    Prof pr(h, OZK_KIND_OTHER, 0.0, 0.0);
    launch_kkr_step(-1, 0, nleaves, nsolves, dn, Mp, b, W, w, dinv, t, h->stream);
  }
  GjParams gj{};
  gj.D = t.D; gj.ldd = t.ldd; gj.nb = t.nbv;
  gj.R = reinterpret_cast<const double2* const*>(t0); gj.ldr = t.nbv;
  gj.X = reinterpret_cast<double2* const*>(tau); gj.ldx = t.nbv; gj.nrhs = b; gj.status = h->d_status;
  {
    Prof pr(h, OZK_KIND_GJ, 16.0 * b * b * b * nsolves, 48.0 * b * b * nsolves);
    launch_gj(gj, b, b, nsolves, h->stream);
  }
  return cuda_check(cudaGetLastError(), "kkr_tau00_batched launches");
}

// ---- slice-count selector
ozk_status_t ozk_selector_init(ozk_handle_t h, uint64_t seed) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  // He-scaled normals (Box-Muller on a SplitMix64 stream), zero hidden biases, output biases
  // at -8 (the middle of the log10 error range the outputs predict)
  std::vector<float> p(SEL_NPARAMS, 0.0f);
  const uint64_t base = sm_base_host(seed, 0x5E1ull);
  auto mix = [](uint64_t z) {
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull; z ^= z >> 31;
    return z;
  };
  uint64_t ctr = 0;
  auto unif = [&]() { return static_cast<double>(mix(base + (++ctr) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53; };
  auto normal = [&]() {
    const double u1 = 1.0 - unif(), u2 = unif();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.141592653589793 * u2);
  };
  const int W1 = 0, W2 = SEL_NH * SEL_NF + SEL_NH, W3 = W2 + SEL_NH * SEL_NH + SEL_NH, B3 = W3 + SEL_NO * SEL_NH;
  for (int i = 0; i < SEL_NH * SEL_NF; ++i) p[W1 + i] = static_cast<float>(normal() * std::sqrt(2.0 / SEL_NF));
  for (int i = 0; i < SEL_NH * SEL_NH; ++i) p[W2 + i] = static_cast<float>(normal() * std::sqrt(2.0 / SEL_NH));
  for (int i = 0; i < SEL_NO * SEL_NH; ++i) p[W3 + i] = static_cast<float>(normal() * std::sqrt(1.0 / SEL_NH));
  for (int o = 0; o < SEL_NO; ++o) p[B3 + o] = -8.0f;
  return sel_upload(h, p.data());
}

ozk_status_t ozk_selector_set_params(ozk_handle_t h, const float* params) {
  if (!h || !params) return set_error(OZK_ERR_ARG, "null argument");
  for (int i = 0; i < SEL_NPARAMS; ++i)
    if (!std::isfinite(params[i])) return set_error(OZK_ERR_ARG, "non-finite selector parameter");
  return sel_upload(h, params);
}

ozk_status_t ozk_selector_get_params(ozk_handle_t h, float* params) {
  if (!h || !params) return set_error(OZK_ERR_ARG, "null argument");
  if (!h->sel_ready) return set_error(OZK_ERR_ARG, "selector has no parameters");
  ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  return cuda_check(cudaMemcpy(params, h->sel_p, sizeof(float) * SEL_NPARAMS, cudaMemcpyDeviceToHost), "read params");
}

static const char kSelMagic[8] = {'O', 'Z', 'K', 'S', 'E', 'L', '1', '\0'};

ozk_status_t ozk_selector_load(ozk_handle_t h, const char* path) {
  if (!h || !path) return set_error(OZK_ERR_ARG, "null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(OZK_ERR_NOFILE, "cannot open selector parameter file");
  char magic[8];
  int32_t np = 0;
  std::vector<float> p(SEL_NPARAMS);
  const bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kSelMagic, 8) == 0 &&
                  std::fread(&np, sizeof(np), 1, f) == 1 && np == SEL_NPARAMS &&
                  std::fread(p.data(), sizeof(float), SEL_NPARAMS, f) == static_cast<size_t>(SEL_NPARAMS);
  std::fclose(f);
  if (!ok) return set_error(OZK_ERR_ARG, "malformed selector parameter file");
  return ozk_selector_set_params(h, p.data());
}

ozk_status_t ozk_selector_save(ozk_handle_t h, const char* path) {
  if (!h || !path) return set_error(OZK_ERR_ARG, "null argument");
  std::vector<float> p(SEL_NPARAMS);
  ozk_status_t st = ozk_selector_get_params(h, p.data());
  if (st) return st;
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(OZK_ERR_NOFILE, "cannot create selector parameter file");
  const int32_t np = SEL_NPARAMS;
  const bool ok = std::fwrite(kSelMagic, 1, 8, f) == 8 && std::fwrite(&np, sizeof(np), 1, f) == 1 &&
                  std::fwrite(p.data(), sizeof(float), SEL_NPARAMS, f) == static_cast<size_t>(SEL_NPARAMS);
  const bool closed = std::fclose(f) == 0;
  return ok && closed ? OZK_OK : set_error(OZK_ERR_NOFILE, "cannot write selector parameter file");
}

ozk_status_t ozk_selector_configure(ozk_handle_t h, double tol, double margin, int flags) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  if (!(tol > 0.0) || !std::isfinite(tol) || !std::isfinite(margin) || (flags & ~OZK_SEL_NO_FALLBACK))
    return set_error(OZK_ERR_ARG, "need tol > 0, finite margin, flags in {0, OZK_SEL_NO_FALLBACK}");
  h->sel_tol = tol;
  h->sel_margin = margin;
  h->sel_flags = flags;
  return OZK_OK;
}

ozk_status_t ozk_selector_features(ozk_handle_t h, char transa, char transb, int m, int n, int k, const void* A,
                                   int lda, const void* B, int ldb, uint64_t probe_seed, float* features) {
  if (!h || !A || !B || !features) return set_error(OZK_ERR_ARG, "null argument");
  OpFlags oa, ob;
  if (!parse_op(transa, &oa) || !parse_op(transb, &ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  if (m < 1 || n < 1 || k < 1) return set_error(OZK_ERR_ARG, "features need m, n, k >= 1");
  ozk_status_t st = check_dims(oa, ob, m, n, k, lda, ldb, m);
  if (st) return st;
  SelScratch s;
  st = sel_scratch(h, m, n, k, false, &s);
  if (st) return st;
  st = sel_features(h, oa, ob, m, n, k, static_cast<const double2*>(A), lda, static_cast<const double2*>(B), ldb,
                    probe_seed, s);
  if (st) return st;
  return cuda_check(cudaMemcpyAsync(features, s.f, sizeof(float) * SEL_NF, cudaMemcpyDeviceToDevice, h->stream),
                    "copy features");
}

ozk_status_t ozk_selector_predict(ozk_handle_t h, int N, const float* X, float* Y) {
  if (!h || (N > 0 && (!X || !Y))) return set_error(OZK_ERR_ARG, "null argument");
  if (N < 0) return set_error(OZK_ERR_ARG, "negative N");
  if (!h->sel_ready) return set_error(OZK_ERR_ARG, "selector has no parameters");
  launch_mlp_forward(h->sel_p, X, N, nullptr, nullptr, Y, h->stream);
  return cuda_check(cudaGetLastError(), "selector forward launch");
}

// training scratch for N samples: Z1, Z2, dZ2, dZ1 (N x 64), Y, dY (N x 8), loss
struct SelTrain { float *Z1, *Z2, *dZ2, *dZ1, *Y, *dY; double* loss; };
static ozk_status_t sel_train_scratch(ozk_context* h, int N, SelTrain* t) {
  const size_t a = align_up(sizeof(float) * size_t(N) * SEL_NH, 256), b = align_up(sizeof(float) * size_t(N) * SEL_NO, 256);
  ozk_status_t st = ensure_sel_ws(h, 4 * a + 2 * b + 256);
  if (st) return st;
  uint8_t* p = static_cast<uint8_t*>(h->sel_ws);
  t->Z1 = reinterpret_cast<float*>(p); t->Z2 = reinterpret_cast<float*>(p + a);
  t->dZ2 = reinterpret_cast<float*>(p + 2 * a); t->dZ1 = reinterpret_cast<float*>(p + 3 * a);
  t->Y = reinterpret_cast<float*>(p + 4 * a); t->dY = reinterpret_cast<float*>(p + 4 * a + b);
  t->loss = reinterpret_cast<double*>(p + 4 * a + 2 * b);
  return OZK_OK;
}

ozk_status_t ozk_selector_train_step(ozk_handle_t h, int N, const float* X, const float* T, float lr, double* loss) {
  if (!h || !X || !T) return set_error(OZK_ERR_ARG, "null argument");
  if (N < 1 || !(lr > 0.0f)) return set_error(OZK_ERR_ARG, "need N >= 1 and lr > 0");
  if (!h->sel_ready) return set_error(OZK_ERR_ARG, "selector has no parameters");
  SelTrain t;
  ozk_status_t st = sel_train_scratch(h, N, &t);
  if (st) return st;
  h->sel_t += 1;
  float* P = h->sel_p;
  launch_mlp_train(P, P + 3 * SEL_NPARAMS, P + SEL_NPARAMS, P + 2 * SEL_NPARAMS, h->sel_t, lr, X, T, N, t.Z1, t.Z2,
                   t.Y, t.dY, t.dZ2, t.dZ1, t.loss, h->stream);
  st = cuda_check(cudaGetLastError(), "selector training launches");
  if (st || !loss) return st;
  st = cuda_check(cudaMemcpyAsync(loss, t.loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read loss");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
}

ozk_status_t ozk_selector_gradient(ozk_handle_t h, int N, const float* X, const float* T, float* grad) {
  if (!h || !X || !T || !grad) return set_error(OZK_ERR_ARG, "null argument");
  if (N < 1) return set_error(OZK_ERR_ARG, "need N >= 1");
  if (!h->sel_ready) return set_error(OZK_ERR_ARG, "selector has no parameters");
  SelTrain t;
  ozk_status_t st = sel_train_scratch(h, N, &t);
  if (st) return st;
  launch_mlp_grad_only(h->sel_p, grad, X, T, N, t.Z1, t.Z2, t.Y, t.dY, t.dZ2, t.dZ1, h->stream);
  return cuda_check(cudaGetLastError(), "selector gradient launches");
}

ozk_status_t ozk_selector_last(ozk_handle_t h, ozk_selector_info* info) {
  if (!h || !info) return set_error(OZK_ERR_ARG, "null argument");
  *info = h->sel_last;
  return OZK_OK;
}

ozk_status_t ozk_rel_diff(ozk_handle_t h, int m, int n, const void* X, int ldx, const void* Y, int ldy, double* rel) {
  if (!h || !X || !Y || !rel) return set_error(OZK_ERR_ARG, "null argument");
  if (m < 1 || n < 1 || ldx < m || ldy < m) return set_error(OZK_ERR_ARG, "need m, n >= 1 and ld >= m");
  ozk_status_t st = ensure_sel_ws(h, align_up(sizeof(double) * 2 * size_t(n), 256) + 256);
  if (st) return st;
  double* part = static_cast<double*>(h->sel_ws);
  double* out = reinterpret_cast<double*>(static_cast<uint8_t*>(h->sel_ws) + align_up(sizeof(double) * 2 * size_t(n), 256));
  launch_rel_diff(m, n, static_cast<const double2*>(X), ldx, static_cast<const double2*>(Y), ldy, part, out, h->stream);
  st = cuda_check(cudaGetLastError(), "rel diff launches");
  if (st) return st;
  st = cuda_check(cudaMemcpyAsync(rel, out, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read rel diff");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
}

static std::vector<int> tune_key(int nsolves, const int* n, int b, int S) {
  std::vector<int> key(n, n + nsolves);
  key.push_back(b);
  key.push_back(S);
  return key;
}

// Times the batched solve on scratch copies of diagonally dominant test matrices of the given
// sizes for every (W, w) candidate (one warm and one timed run each); the index of the fastest
// into *best and the times into times[] (may be null).
static ozk_status_t autotune_impl(ozk_context* h, int nsolves, const int* n, int b, int S,
                                  const std::vector<std::pair<int, int>>& cands, int* best, float* times) {
  if (capturing(h->stream)) return set_error(OZK_ERR_CAPTURE, "autotuning times launches and cannot be captured");
  size_t total = 0;
  for (int i = 0; i < nsolves; ++i) {
    if (n[i] <= 0 || n[i] % b) return set_error(OZK_ERR_ARG, "every n[i] must be a positive multiple of b");
    total += static_cast<size_t>(n[i]) * n[i];
  }
  // scratch: diagonally dominant test matrices (timings do not depend on the values, but the
  // pivot blocks must be regular), a t_0, the outputs and the pointer arrays
  void* mem = nullptr;
  const size_t mbytes = align_up(sizeof(double2) * total, 256);
  const size_t tbytes = align_up(sizeof(double2) * static_cast<size_t>(b) * b * (nsolves + 1), 256);
  const size_t pbytes = align_up(3 * sizeof(void*) * static_cast<size_t>(nsolves), 256);
  ozk_status_t st = cuda_check(cudaMalloc(&mem, mbytes + tbytes + pbytes), "cudaMalloc(autotune scratch)");
  if (st) return st;
  double2* Mall = static_cast<double2*>(mem);
  double2* tall = reinterpret_cast<double2*>(static_cast<uint8_t*>(mem) + mbytes);
  void** ptrs = reinterpret_cast<void**>(static_cast<uint8_t*>(mem) + mbytes + tbytes);
  std::vector<void*> hp(3 * static_cast<size_t>(nsolves));
  size_t off = 0;
  for (int i = 0; i < nsolves; ++i) {
    hp[i] = Mall + off;
    off += static_cast<size_t>(n[i]) * n[i];
    hp[nsolves + i] = tall;                                           // shared t_0
    hp[2 * static_cast<size_t>(nsolves) + i] = tall + static_cast<size_t>(b) * b * (i + 1);
  }
  const int* dn = nullptr;
  st = size_table(h, std::vector<int>(n, n + nsolves), &dn);
  if (!st) st = cuda_check(cudaMemcpyAsync(ptrs, hp.data(), sizeof(void*) * hp.size(), cudaMemcpyHostToDevice, h->stream),
                           "upload autotune pointers");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!st) st = cuda_check(cudaEventCreate(&e0), "cudaEventCreate");
  if (!st) st = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  std::vector<float> ms_all(cands.size(), 0.0f);
  *best = -1;
  const bool prof = h->prof;
  h->prof = false;                                                    // tuning runs are not profiled
  for (size_t c = 0; c < cands.size() && !st; ++c) {
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && !st; ++rep) {                        // warm run, then the timed one
      launch_fill_test(reinterpret_cast<double2* const*>(ptrs), dn, nsolves, b, tall, h->stream);
      cudaEventRecord(e0, h->stream);
      st = tau00_batched_impl(h, nsolves, n, b, ptrs, reinterpret_cast<const void* const*>(ptrs + nsolves),
                              ptrs + 2 * nsolves, S, cands[c].first, cands[c].second);
      cudaEventRecord(e1, h->stream);
      if (!st) st = cuda_check(cudaEventSynchronize(e1), "cudaEventSynchronize");
      if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    }
    if (st) break;
    if (times) times[c] = ms;
    ms_all[c] = ms;
  }
  if (!st && !cands.empty()) {
    // the smallest (W, w) among the candidates within 1 % of the fastest: timing noise between
    // near-equal pairs does not decide, and the narrower panel needs less workspace
    const float fastest = *std::min_element(ms_all.begin(), ms_all.end());
    for (size_t c = 0; c < cands.size(); ++c)
      if (ms_all[c] <= 1.01f * fastest && (*best < 0 || cands[c] < cands[*best])) *best = static_cast<int>(c);
  }
  h->prof = prof;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(h->stream);
  cudaFree(mem);
  return st;
}

ozk_status_t kkr_tau00_autotune(ozk_handle_t h, int nsolves, const int* n, int b, int S, int* nb_best, float* times) {
  if (!h || !n || !nb_best) return set_error(OZK_ERR_ARG, "null argument");
  if (nsolves < 1 || S < 1 || b < 1 || b > 64) return set_error(OZK_ERR_ARG, "need nsolves >= 1, S >= 1, 1 <= b <= 64");
  std::vector<std::pair<int, int>> cands;
  for (int nb = b; nb <= GJINV_MAX; nb += b) cands.push_back({nb, nb});
  int best = -1;
  ozk_status_t st = autotune_impl(h, nsolves, n, b, S, cands, &best, times);
  if (st) return st;
  h->tuned_nb[tune_key(nsolves, n, b, S)] = cands[best];
  *nb_best = cands[best].first;
  return OZK_OK;
}

ozk_status_t kkr_tau00_autotune_panels(ozk_handle_t h, int nsolves, const int* n, int b, int S, int* W_best,
                                       int* w_best, float* times, int* cand, int cap, int* ncand) {
  if (!h || !n || !W_best || !w_best) return set_error(OZK_ERR_ARG, "null argument");
  if (nsolves < 1 || S < 1 || b < 1 || b > 64) return set_error(OZK_ERR_ARG, "need nsolves >= 1, S >= 1, 1 <= b <= 64");
  // whole-panel pivot blocks nb = b, 2b, ... <= 112, then panels of 2 to 4 leaves (one matrix:
  // up to 8, its inverses having the GPU to themselves) of every leaf width w (a multiple of
  // b) from 32 to 96
  std::vector<std::pair<int, int>> cands;
  for (int nb = b; nb <= GJINV_MAX; nb += b) cands.push_back({nb, nb});
  const int gmax = nsolves == 1 ? 8 : 4;
  for (int w = b; w <= std::min(96, GJINV_MAX); w += b) {
    if (w < 32) continue;
    for (int g = 2; g <= gmax; ++g)
      if (g * w <= OZK_PANEL_MAX) cands.push_back({g * w, w});
  }
  if (ncand) *ncand = static_cast<int>(cands.size());
  if (times && static_cast<int>(cands.size()) > cap) return set_error(OZK_ERR_ARG, "times/cand arrays too short");
  int best = -1;
  ozk_status_t st = autotune_impl(h, nsolves, n, b, S, cands, &best, times);
  if (st) return st;
  if (cand)
    for (size_t c = 0; c < cands.size(); ++c) { cand[2 * c] = cands[c].first; cand[2 * c + 1] = cands[c].second; }
  h->tuned_nb[tune_key(nsolves, n, b, S)] = cands[best];
  *W_best = cands[best].first;
  *w_best = cands[best].second;
  return OZK_OK;
}

// S = 0 for a batched solve.  One slice count serves every GEMM launch of the call (a launch
// covers all solves), so it is chosen from a sample of up to 8 solves: the largest, the
// smallest and solves spread over the call.  For each sampled solve the selector picks S for
// the leading block (at most 512 x 512 outputs) of its first trailing update (L panel
// M[0:p, p:q] times U panel M[p:q, 0:p] of the unfactored M, q = n_i, p = max(q - w, b)); the
// call takes the largest pick.  Every sampled product is then computed at that S and checked
// with the probes (recorded on the device, read once); if any check fails the call runs at
// S = 10.  The block bounds the check, whose binary64 probe products cost O(outputs x probes).
constexpr int SEL_BATCH_SAMPLES = 8;
constexpr int SEL_BATCH_BLOCK = 512;
static ozk_status_t select_S_for_solves(ozk_context* h, int nsolves, void* const* M, const int* n, int b, int w,
                                        int* S_out) {
  if (!h->sel_ready)
    return set_error(OZK_ERR_ARG, "S = 0 needs selector parameters (ozk_selector_init, _load or _set_params)");
  if (capturing(h->stream)) return set_error(OZK_ERR_CAPTURE, "S = 0 reads the selector's choice and cannot be captured");
  std::vector<void*> mp(nsolves);
  ozk_status_t st = cuda_check(cudaMemcpy(mp.data(), M, sizeof(void*) * nsolves, cudaMemcpyDeviceToHost), "read M");
  if (st) return st;
  std::vector<int> pick;
  auto add = [&](int i) {
    if (n[i] > b && std::find(pick.begin(), pick.end(), i) == pick.end()) pick.push_back(i);
  };
  add(static_cast<int>(std::max_element(n, n + nsolves) - n));
  add(static_cast<int>(std::min_element(n, n + nsolves) - n));
  for (int j = 0; j < SEL_BATCH_SAMPLES && static_cast<int>(pick.size()) < SEL_BATCH_SAMPLES; ++j)
    add(static_cast<int>((static_cast<long long>(j) * nsolves) / SEL_BATCH_SAMPLES));
  ozk_selector_info info{};
  if (pick.empty()) {
    info.S_selected = info.S_used = SEL_SMAX;
    h->sel_last = info;
    *S_out = SEL_SMAX;
    return OZK_OK;
  }
  const int wp = w > 0 ? w : 64;
  auto gemm_of = [&](int i) {
    EmuGemm g;
    const int q = n[i], p = std::max(q - wp, b);
    const double2* Mi = static_cast<const double2*>(mp[i]);
    g.oa = {0, 0}; g.ob = {0, 0}; g.batch = 1;
    const int pb = std::min(p, SEL_BATCH_BLOCK);
    g.mmax = g.m = pb; g.nmax = g.n = pb; g.kmax = g.k = q - p;
    g.A = Mi + static_cast<long long>(p) * q; g.lda = q; g.B = Mi + p; g.ldb = q;
    g.ar = 1; g.ai = 0; g.br = 0; g.bi = 0;
    g.pair_mode = OZK_PAIRS_TRI;
    return g;
  };
  int S = SEL_SMIN;
  for (int i : pick) {
    const EmuGemm g = gemm_of(i);
    SelScratch sc;
    st = sel_scratch(h, g.m, g.n, g.k, false, &sc);
    if (!st) {
      info.probe_seed = h->sel_seed + h->sel_calls++;
      st = sel_features(h, g.oa, g.ob, g.m, g.n, g.k, g.A, g.lda, g.B, g.ldb, info.probe_seed, sc);
    }
    if (st) return st;
    launch_mlp_forward(h->sel_p, sc.f, 1, nullptr, nullptr, sc.Y, h->stream);
    launch_choose(sc.Y, static_cast<float>(std::log10(h->sel_tol) - h->sel_margin), sc.aux, h->stream);
    SelAux aux;
    st = read_aux(h, sc.aux, &aux);
    if (st) return st;
    S = std::max(S, aux.S);
    if (i == pick.front())
      for (int o = 0; o < SEL_NO; ++o) info.predicted_log10_err[o] = aux.pred[o];
  }
  info.S_selected = info.S_used = S;
  // the checks: each sampled product at S into the scratch D (the GEMM workspace at offset 0 is
  // free before the solve starts), recorded on the device
  if (!h->sel_rec) {
    st = cuda_check(cudaMalloc(&h->sel_rec, sizeof(SelDefer)), "cudaMalloc(check record)");
    if (st) { h->sel_rec = nullptr; return st; }
  }
  SelDefer* rec = h->sel_rec;
  SelDefer r{};
  st = cuda_check(cudaMemsetAsync(rec, 0, sizeof(SelDefer), h->stream), "clear check record");
  for (int i : pick) {
    if (st) return st;
    EmuGemm g = gemm_of(i);
    SelScratch sc;
    st = sel_scratch(h, g.m, g.n, g.k, true, &sc);
    if (st) return st;
    st = sel_features(h, g.oa, g.ob, g.m, g.n, g.k, g.A, g.lda, g.B, g.ldb, h->sel_seed + h->sel_calls++, sc);
    if (st) return st;
    g.C = sc.D; g.ldc = g.m; g.S = S; g.mode = -1;
    st = run_emulated(h, g, 0);
    if (st) return st;
    launch_gemv(sc.D, g.m, g.m, g.n, 0, sc.X, nullptr, g.n, sc.Wh, sc.Wl, sc.part, nullptr, 0, h->stream, true);
    launch_residual(sc.Wh, sc.Wl, sc.zh, sc.zl, g.m, sc.aux, reinterpret_cast<double*>(sc.part), h->stream);
    launch_defer_check(sc.aux, S, false, 0.5 * h->sel_tol, rec, h->stream);
    st = cuda_check(cudaGetLastError(), "check launches");
  }
  if (!st) st = cuda_check(cudaMemcpyAsync(&r, rec, sizeof(SelDefer), cudaMemcpyDeviceToHost, h->stream), "read record");
  if (!st) st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  info.gemms = static_cast<int>(pick.size());
  info.S_count[S - SEL_SMIN] = info.gemms;
  info.residual = info.residual_selected = r.max_resid;
  info.residual_ok = r.failed ? 0 : 1;
  if (r.failed) {
    if (h->sel_flags & OZK_SEL_NO_FALLBACK) {
      h->sel_last = info;
      return set_error(OZK_ERR_RESIDUAL, "a sampled product failed its residual check and fallback is disabled");
    }
    info.S_used = SEL_SMAX;
    info.fallback = 1;
  }
  h->sel_last = info;
  *S_out = info.S_used;
  return OZK_OK;
}

ozk_status_t kkr_tau00_batched_panels(ozk_handle_t h, int nsolves, const int* n, int b, void* const* M,
                                      const void* const* t0, void* const* tau, int S, int W, int w) {
  if (!h || !n) return set_error(OZK_ERR_ARG, "null argument");
  if (S == 0 && nsolves > 0) {
    if (!M || n[0] <= 0) return set_error(OZK_ERR_ARG, "bad solve 0");
    ozk_status_t st = select_S_for_solves(h, nsolves, M, n, b, w > 0 ? w : W, &S);
    if (st) return st;
  }
  if (W == 0 && nsolves > 0 && S < 0) W = w = std::min(GJINV_MAX, (32 + b - 1) / b * b);   // binary64: as kkr_tau00
  if (W == 0 && nsolves > 0) {
    auto it = h->tuned_nb.find(tune_key(nsolves, n, b, S));
    if (it != h->tuned_nb.end()) {
      W = it->second.first;
      w = it->second.second;
    } else {
      ozk_status_t st = kkr_tau00_autotune_panels(h, nsolves, n, b, S, &W, &w, nullptr, nullptr, 0, nullptr);
      if (st) return st;
    }
  }
  return tau00_batched_impl(h, nsolves, n, b, M, t0, tau, S, W, w);
}

ozk_status_t kkr_tau00_batched(ozk_handle_t h, int nsolves, const int* n, int b, void* const* M, const void* const* t0,
                               void* const* tau, int S, int nb) {
  if (nb > GJINV_MAX) return set_error(OZK_ERR_ARG, "nb <= 112 (the pivot block is held in shared memory)");
  return kkr_tau00_batched_panels(h, nsolves, n, b, M, t0, tau, S, nb, nb);
}

ozk_status_t kkr_contour_trace(ozk_handle_t h, int nsolves, int b, const void* const* tau, const double* w,
                               double* traces, double* integral) {
  if (!h || !tau || !w || !integral) return set_error(OZK_ERR_ARG, "null argument");
  if (nsolves < 1 || b < 1) return set_error(OZK_ERR_ARG, "need nsolves >= 1 and b >= 1");
  const size_t wb = align_up(sizeof(double2) * nsolves, 256);
  ozk_status_t st = ensure_sel_ws(h, 3 * wb + 256);
  if (st) return st;
  uint8_t* base = static_cast<uint8_t*>(h->sel_ws);
  double2* dw = reinterpret_cast<double2*>(base);
  double2* tr = reinterpret_cast<double2*>(base + wb);
  double2* out = reinterpret_cast<double2*>(base + 2 * wb);
  st = cuda_check(cudaMemcpyAsync(dw, w, sizeof(double2) * nsolves, cudaMemcpyHostToDevice, h->stream), "upload weights");
  if (st) return st;
  launch_contour_trace(reinterpret_cast<const double2* const*>(tau), nsolves, b, dw, tr, out, h->stream);
  st = cuda_check(cudaGetLastError(), "contour trace launches");
  if (st) return st;
  if (traces) {
    st = cuda_check(cudaMemcpyAsync(traces, tr, sizeof(double2) * nsolves, cudaMemcpyDeviceToHost, h->stream), "read traces");
    if (st) return st;
  }
  st = cuda_check(cudaMemcpyAsync(integral, out, sizeof(double2), cudaMemcpyDeviceToHost, h->stream), "read integral");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
}

ozk_status_t ozk_profile_begin(ozk_handle_t h) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  h->recs.clear();
  h->pool_used = 0;
  h->prof = true;
  return OZK_OK;
}

ozk_status_t ozk_profile_end(ozk_handle_t h, uint64_t* launches, double* ms, double* flops, double* bytes) {
  if (!h || !launches || !ms || !flops || !bytes) return set_error(OZK_ERR_ARG, "null argument");
  h->prof = false;
  ozk_status_t st = cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st) return st;
  for (int k = 0; k < OZK_KERNEL_KINDS; ++k) { launches[k] = 0; ms[k] = 0; flops[k] = 0; bytes[k] = 0; h->prof_moved[k] = 0; }
  for (const ProfRec& r : h->recs) {
    float t = 0.f;
    st = cuda_check(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
    if (st) return st;
    launches[r.kind] += 1;
    ms[r.kind] += t;
    flops[r.kind] += r.flops;
    bytes[r.kind] += r.bytes;
    h->prof_moved[r.kind] += r.moved;
  }
  h->recs.clear();
  return OZK_OK;
}

ozk_status_t ozk_selector_log_begin(ozk_handle_t h, float* features, float* targets, int capacity) {
  if (!h || !features || !targets || capacity < 1) return set_error(OZK_ERR_ARG, "need buffers and capacity >= 1");
  h->sel_log_f = features;
  h->sel_log_t = targets;
  h->sel_log_cap = capacity;
  h->sel_log_n = 0;
  return OZK_OK;
}

ozk_status_t ozk_selector_log_end(ozk_handle_t h, int* count) {
  if (!h || !count) return set_error(OZK_ERR_ARG, "null argument");
  *count = h->sel_log_n;
  h->sel_log_f = nullptr;
  h->sel_log_t = nullptr;
  h->sel_log_cap = h->sel_log_n = 0;
  return cuda_check(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
}

ozk_status_t ozk_debug_stall_next_gemm(ozk_handle_t h, long long cycles) {
  if (!h) return set_error(OZK_ERR_ARG, "null handle");
  h->stall_next = cycles > 0 ? cycles : 0;
  return OZK_OK;
}

ozk_status_t ozk_profile_moved(ozk_handle_t h, double* moved) {
  if (!h || !moved) return set_error(OZK_ERR_ARG, "null argument");
  for (int k = 0; k < OZK_KERNEL_KINDS; ++k) moved[k] = h->prof_moved[k];
  return OZK_OK;
}


ozk_status_t kkr_build_m_batched(ozk_handle_t h, int batch, const int* L, int b, const void* const* t,
                                 const void* const* G, void* const* M) {
  if (!h || !L || !t || !G || !M) return set_error(OZK_ERR_ARG, "null argument");
  if (batch < 0 || b <= 0) return set_error(OZK_ERR_ARG, "bad size");
  if (batch == 0) return OZK_OK;
  int nmax = 0;
  double nn2 = 0;
  for (int i = 0; i < batch; ++i) {
    if (L[i] <= 0) return set_error(OZK_ERR_ARG, "L[i] must be positive");
    nmax = std::max(nmax, L[i] * b);
    nn2 += static_cast<double>(L[i]) * b * L[i] * b;
  }
  const int* dL = nullptr;
  ozk_status_t st = size_table(h, std::vector<int>(L, L + batch), &dL);
  if (st) return st;
  {
    Prof pr(h, OZK_KIND_BUILD_M, 8.0 * nn2 * b, 32.0 * nn2);
    launch_build_m_batched(dL, b, reinterpret_cast<const double2* const*>(t), reinterpret_cast<const double2* const*>(G),
                           reinterpret_cast<double2* const*>(M), nmax, batch, h->stream);
  }
  return cuda_check(cudaGetLastError(), "build_m_batched launch");
}

}  // extern "C"

// --------------------------------------------------------------------- allocation-free ZGEMM
// Some callers cannot allocate device memory at the point where they need a GEMM: code that
// runs while a CUDA graph is being captured (cudaMalloc is not a capturable operation), code
// inside a memory-pool-managed framework that forbids allocations outside its allocator, or
// a host thread holding a lock that a device allocation would contend for.  For them this
// entry point runs the same emulated ZGEMM with its scratch (slice planes and exponents) in a
// statically sized device array of this file, so it allocates nothing.  The array is part of
// the library image: every GPU that loads the library keeps OZK_NOALLOC_SCRATCH_BYTES of it
// until the process exits.  All calls share it, so calls that may overlap on the GPU (other
// streams, other threads) race and must be serialised by the caller.
static __device__ __align__(256) unsigned char g_noalloc_scratch[OZK_NOALLOC_SCRATCH_BYTES];
static __device__ int g_noalloc_status;

namespace {
constexpr int kMaxDevices = 64;
struct NoallocAddr { void* scratch; int* status; };
std::atomic<const NoallocAddr*> g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the static scratch for the current device, looked up once per device
// (the name is only a host-side stand-in for the device symbol).  Host threads that make their
// first call at the same time serialise on a mutex; later calls read the published addresses
// without locking.
ozk_status_t noalloc_setup(int dev, void** scratch, int** status) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(OZK_ERR_ARG, "device index out of range for the static scratch");
  const NoallocAddr* a = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    a = g_noalloc_addr[dev].load(std::memory_order_relaxed);
    if (!a) {
      void* p = nullptr;
      void* s = nullptr;
      ozk_status_t st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
      if (st) return st;
      st = cuda_check(cudaGetSymbolAddress(&s, g_noalloc_status), "cudaGetSymbolAddress(status)");
      if (st) return st;
      a = new NoallocAddr{p, static_cast<int*>(s)};      // kept until the process exits
      g_noalloc_addr[dev].store(a, std::memory_order_release);
    }
  }
  *scratch = a->scratch;
  *status = a->status;
  return OZK_OK;
}
}  // namespace

extern "C" ozk_status_t ozaki_zgemm_noalloc(void* stream, char transa, char transb, int m, int n, int k,
                                           const double* alpha, const void* A, int lda, const void* B, int ldb,
                                           const double* beta, void* C, int ldc, int S, int pair_mode,
                                           int* device_status) {
  if (!alpha || !beta) return set_error(OZK_ERR_ARG, "null argument");
  EmuGemm g;
  if (!parse_op(transa, &g.oa) || !parse_op(transb, &g.ob)) return set_error(OZK_ERR_ARG, "bad trans flag");
  ozk_status_t st = check_dims(g.oa, g.ob, m, n, k, lda, ldb, ldc);
  if (st) return st;
  if (pair_mode != OZK_PAIRS_TRI && pair_mode != OZK_PAIRS_FULL) return set_error(OZK_ERR_ARG, "bad pair mode");
  g.batch = 1; g.mmax = g.m = m; g.nmax = g.n = n; g.kmax = g.k = k;
  g.A = static_cast<const double2*>(A); g.lda = lda;
  g.B = static_cast<const double2*>(B); g.ldb = ldb;
  g.C = static_cast<double2*>(C); g.ldc = ldc;
  g.ar = alpha[0]; g.ai = alpha[1]; g.br = beta[0]; g.bi = beta[1];
  g.S = S; g.pair_mode = pair_mode;
  const bool trivial = (m == 0 || n == 0 || k == 0 || (alpha[0] == 0.0 && alpha[1] == 0.0));
  if (!trivial) {
    GemmPlan P;
    st = plan_gemm(g, &P);
    if (st) return st;
    if (P.total > OZK_NOALLOC_SCRATCH_BYTES)
      return set_error(OZK_ERR_ARG, "ozaki_zgemm_noalloc: problem needs more scratch than OZK_NOALLOC_SCRATCH_BYTES "
                                    "(use ozaki_zgemm with a handle)");
  }
  int dev = 0;
  st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st) return st;
  void* scratch = nullptr;
  int* status = nullptr;
  st = noalloc_setup(dev, &scratch, &status);
  if (st) return st;
  // a context on the stack whose workspace is the static scratch (it owns nothing; run_emulated
  // never grows the workspace because the size was checked above)
  ozk_context ctx;
  ctx.device = dev;
  ctx.stream = static_cast<cudaStream_t>(stream);
  ctx.d_status = device_status ? device_status : status;
  ctx.ws = scratch;
  ctx.ws_bytes = OZK_NOALLOC_SCRATCH_BYTES;
  if (m == 0 || n == 0) return OZK_OK;
  if (trivial) {
    if (beta[0] == 1.0 && beta[1] == 0.0) return OZK_OK;
    launch_scale(m, n, static_cast<double2*>(C), ldc, beta[0], beta[1], ctx.stream);
    return cuda_check(cudaGetLastError(), "scale launch");
  }
  return run_emulated(&ctx, g);
}
