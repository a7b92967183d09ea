// Host side of the C ABI declared in include/bloomgb.h: argument checks,
// layout resolution, kernel dispatch, L2 persistence and the host-buffer
// pipeline.  Every compute step runs in the kernels of sbf_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "bloomgb.h"
#include "host_stage.h"
#include "registry.h"

namespace bloomgb {
constexpr int kMaxBlockThreadsHost = 512;  // matches kMaxBlockThreads of the kernels
}

using namespace bloomgb;

namespace {

thread_local std::string g_last_error;

bf_status fail(bf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

bf_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return BF_ECUDA;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

struct Registry {
  std::vector<KernelEntry> sbf;
  std::vector<GupsEntry> gups;
};

const Registry& registry() {
  static const Registry r = [] {
    Registry reg;
#define BLOOMGB_REGISTER(B, S) register_B##B##_S##S(reg.sbf);
    BLOOMGB_GEOMETRIES(BLOOMGB_REGISTER)
#undef BLOOMGB_REGISTER
    register_gups(reg.gups);
    register_expand(reg.sbf);
    return reg;
  }();
  return r;
}

const KernelEntry* find_sbf(int op, const bf_params& p, const bf_layout& l) {
  for (const auto& e : registry().sbf) {
    if (e.op == op && e.B == static_cast<int>(p.block_bits) && e.S == static_cast<int>(p.word_bits) &&
        e.K == static_cast<int>(p.k) && e.theta == static_cast<int>(l.cg) &&
        e.phi == static_cast<int>(l.phi) && e.kpt == static_cast<int>(l.kpt) && e.z == 0 &&
        e.salts == static_cast<int>(p.salts))
      return &e;
  }
  return nullptr;
}

const KernelEntry* find_csbf(int op, const bf_params& p, const bf_layout& l, uint32_t z) {
  for (const auto& e : registry().sbf) {
    if (e.op == op && e.B == static_cast<int>(p.block_bits) && e.S == static_cast<int>(p.word_bits) &&
        e.K == static_cast<int>(p.k) && e.z == static_cast<int>(z) && e.theta == static_cast<int>(l.cg) &&
        e.kpt == static_cast<int>(l.kpt))
      return &e;
  }
  return nullptr;
}

const GupsEntry* find_gups(int mode, uint32_t unit, uint32_t kpt) {
  for (const auto& e : registry().gups)
    if (e.mode == mode && e.unit_bytes == static_cast<int>(unit) && e.kpt == static_cast<int>(kpt)) return &e;
  return nullptr;
}

// Resident CTAs per SM for a kernel at a CTA size (cached per device).
std::mutex g_occ_mu;
std::unordered_map<std::string, int> g_occ;

bf_status resident_ctas(const void* fn, int threads, int device, int* out) {
  char key[96];
  std::snprintf(key, sizeof key, "%p/%d/%d", fn, threads, device);
  {
    std::lock_guard<std::mutex> g(g_occ_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
      *out = it->second;
      return BF_OK;
    }
  }
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (n < 1) return fail(BF_EINVAL, "kernel cannot run at this CTA size");
  std::lock_guard<std::mutex> g(g_occ_mu);
  g_occ[key] = n;
  *out = n;
  return BF_OK;
}

bf_status sm_count(int device, int* out) {
  cudaError_t e = cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, device);
  return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
}

// grid: at most the resident capacity (a persistent, grid-stride launch),
// and no more CTAs than there are tiles of work.
bf_status resolve_grid(const void* fn, int device, uint32_t threads, uint32_t grid_req, uint64_t n,
                       uint32_t kpt, uint32_t* grid_out) {
  uint64_t tiles = (n + 32ull * kpt - 1) / (32ull * kpt);
  uint64_t ctas_needed = (tiles + threads / 32 - 1) / (threads / 32);
  uint64_t g = grid_req;
  if (g == 0) {
    int sms = 0, per_sm = 0;
    bf_status s = sm_count(device, &sms);
    if (s != BF_OK) return s;
    s = resident_ctas(fn, static_cast<int>(threads), device, &per_sm);
    if (s != BF_OK) return s;
    g = static_cast<uint64_t>(sms) * per_sm;
  }
  g = std::min<uint64_t>(g, std::max<uint64_t>(ctas_needed, 1));
  g = std::min<uint64_t>(g, 0x7FFFFFFFull);
  *grid_out = static_cast<uint32_t>(g);
  return BF_OK;
}

}  // namespace

namespace bloomgb {
const KernelEntry* find_kernel(int op, int block_bits, int word_bits, int k, int theta, int phi, int kpt, int z,
                               int salts) {
  for (const auto& e : registry().sbf)
    if (e.op == op && e.B == block_bits && e.S == word_bits && e.K == k && e.theta == theta && e.phi == phi &&
        e.kpt == kpt && e.z == z && e.salts == salts)
      return &e;
  return nullptr;
}
int kernel_resident_ctas(const void* fn, int threads, int device) {
  int n = 0;
  return resident_ctas(fn, threads, device, &n) == BF_OK ? n : 0;
}
}  // namespace bloomgb

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

constexpr int kPipelineDepth = 3;

}  // namespace

struct bf_filter {
  bf_params p{};
  void* words = nullptr;
  uint64_t nbytes = 0;
  bool owned = false;
  int device = 0;
  bf_layout layout[2]{};
  const KernelEntry* entry[2]{};
  // host-buffer pipeline
  uint64_t chunk_keys = 1ull << 24;
  void* staging = nullptr;  // kPipelineDepth slots of slot_bytes(chunk_keys)
  cudaStream_t pipe[kPipelineDepth]{};
  cudaEvent_t ev_start = nullptr;
  // construction from host-resident keys: record inserts on their own stream
  cudaStream_t rec_stream = nullptr;
  cudaEvent_t ev_part[2]{};
  cudaEvent_t ev_rec[2]{};
  cudaEvent_t ev_done[kPipelineDepth]{};
  // slice-partitioned passes over host buffers staged through device memory:
  // two staging slots (keys, then results), a copy-in stream (highest
  // priority) and a copy-out stream
  void* hstage = nullptr;
  uint64_t hstage_bytes = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_copied[2]{};    // slot's keys are on the device
  cudaEvent_t ev_consumed[2]{};  // slot's keys have been partitioned
  cudaEvent_t ev_computed[2]{};  // slot's results are ready
  cudaEvent_t ev_drained[2]{};   // slot's results are on the host
  int host_access = 0;  // bf_host_mode: BF_HOST_AUTO, BF_HOST_STAGED or BF_HOST_DIRECT
  bool l2_window = false;
  // L2-blocked construction
  bf_partition part{BF_PART_AUTO, 24, 1ull << 32, 0, 26, BF_PART_AUTO, 1ull << 28, 0, 0};
  void* part_ws = nullptr;
  uint64_t part_ws_bytes = 0;
  void* look_ws = nullptr;  // slice-partitioned lookup workspace
  uint64_t look_ws_bytes = 0;
  uint64_t l2_bytes = 0;
  uint32_t last_launches = 0;
  uint32_t* status = nullptr;  // device word: kStatus* bits of failed index checks
  // per-phase timing of the last call (bf_set_timing): event pairs around
  // each group of launches, on the stream the group runs on
  struct Seg {
    int phase;
    cudaEvent_t a, b;
    uint32_t launches;
  };
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Seg> segs;
};

namespace {

// groups of a cache-sectorized filter, or 0 for the sectorized one (z = s is
// the sectorized filter too: one word per group)
uint32_t csbf_groups(const bf_params& p) {
  const uint32_t s = p.block_bits / p.word_bits;
  return (p.groups == 0 || p.groups == s) ? 0 : p.groups;
}

bf_status check_params(const bf_params* p) {
  if (!p) return fail(BF_EINVAL, "params is NULL");
  if (p->num_blocks == 0) return fail(BF_EINVAL, "num_blocks must be >= 1");
  if (p->word_bits != 32 && p->word_bits != 64) return fail(BF_EINVAL, "word_bits must be 32 or 64");
  if (!is_pow2(p->block_bits) || p->block_bits < p->word_bits || p->block_bits > 1024)
    return fail(BF_EINVAL, "block_bits must be a power of two in [word_bits, 1024]");
  const uint32_t s = p->block_bits / p->word_bits;
  if (p->groups > s || (p->groups && s % p->groups != 0))
    return fail(BF_EINVAL, "groups must divide s = block_bits/word_bits");
  const uint32_t z = csbf_groups(*p);
  if (z == 0) {
    if (p->k < s || p->k % s != 0 || p->k > 64)
      return fail(BF_EINVAL, "k must be a multiple of s = block_bits/word_bits, s <= k <= 64");
  } else {
    if (p->k < z || p->k % z != 0 || p->k + z > 64)
      return fail(BF_EINVAL, "cache-sectorized: k must be a multiple of groups and k + groups <= 64");
  }
  if (p->num_blocks > (~0ull) / 128) return fail(BF_EINVAL, "num_blocks too large");
  if (p->salts > 1) return fail(BF_EINVAL, "salts must be 0 (default) or 1 (Parquet split-block)");
  if (p->salts == 1 && !(p->block_bits == 256 && p->word_bits == 32 && p->k == 8 && z == 0))
    return fail(BF_EINVAL, "the Parquet salt set needs block_bits 256, word_bits 32, k 8, a sectorized filter");
  return BF_OK;
}

bf_layout default_layout(const bf_params& p, int op) {
  const uint32_t s = p.block_bits / p.word_bits;
  bf_layout l{};
  if (const uint32_t z = csbf_groups(p)) {
    // cache-sectorized: every group's word update in one instruction; lookups one thread per key
    l.cg = op == BF_OP_ADD ? z : 1;
    l.phi = 1;
    l.kpt = op == BF_OP_ADD ? 1 : 2;
  } else if (op == BF_OP_ADD) {
    // Sec. V-B: a fully horizontal layout (Theta = s) coalesces the atomics
    l.cg = s;
    l.phi = 1;
    l.kpt = 1;
  } else {
    // Sec. V-B: lookup favours one thread per 32-byte sector
    uint32_t cg = std::max<uint32_t>(1, p.block_bits / 256);
    l.cg = std::min(cg, s);
    l.phi = s / l.cg;
    l.kpt = 2;
  }
  l.block_threads = 256;
  l.grid_ctas = 0;
  l.flags = 0;
  return l;
}

bf_status resolve_layout(const bf_params& p, int op, const bf_layout* in, bf_layout* out,
                         const KernelEntry** entry) {
  if (op != BF_OP_ADD && op != BF_OP_CONTAINS) return fail(BF_EINVAL, "op must be BF_OP_ADD or BF_OP_CONTAINS");
  const uint32_t s = p.block_bits / p.word_bits;
  const uint32_t z = csbf_groups(p);
  bf_layout d = default_layout(p, op);
  bf_layout l = in ? *in : d;
  if (l.cg == 0) l.cg = d.cg;
  if (l.phi == 0) l.phi = z ? 1 : std::max<uint32_t>(1, s / l.cg);
  if (l.kpt == 0) l.kpt = d.kpt;
  if (l.block_threads == 0) l.block_threads = d.block_threads;
  if (z) {
    if (!is_pow2(l.cg) || z % l.cg != 0 || l.phi != 1)
      return fail(BF_EINVAL, "cache-sectorized layout: cg a power of two dividing groups, phi = 1");
  } else if (!is_pow2(l.cg) || !is_pow2(l.phi) || static_cast<uint64_t>(l.cg) * l.phi > s) {
    return fail(BF_EINVAL, "layout needs powers of two with 1 <= cg*phi <= s");
  }
  if (l.kpt != 1 && l.kpt != 2 && l.kpt != 4) return fail(BF_EINVAL, "kpt must be 1, 2 or 4");
  if (l.block_threads % 32 != 0 || l.block_threads > static_cast<uint32_t>(kMaxBlockThreadsHost))
    return fail(BF_EINVAL, "block_threads must be a multiple of 32 and <= 512");
  if (l.flags & ~(BF_HINT_FILTER_EVICT_LAST | BF_HINT_KEYS_EVICT_NORMAL | BF_HINT_PREFETCH_L2 | BF_HINT_WARP_AGGREGATE))
    return fail(BF_EINVAL, "unknown layout flag");
  const KernelEntry* e = z ? find_csbf(op == BF_OP_ADD ? 9 : 10, p, l, z) : find_sbf(op, p, l);
  if (!e) return fail(BF_EUNSUPPORTED, "no compiled kernel for this geometry and layout");
  *out = l;
  if (entry) *entry = e;
  return BF_OK;
}

// Phase timing: phase_begin records an event before a group of launches,
// phase_end one after it (same stream) and keeps the pair for bf_get_timing.
struct PhaseMark {
  int phase = -1;
  cudaEvent_t a = nullptr;
};

cudaEvent_t pool_event(bf_filter* f) {
  if (f->ev_used == f->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    f->ev_pool.push_back(e);
  }
  return f->ev_pool[f->ev_used++];
}

PhaseMark phase_begin(const bf_filter* fc, cudaStream_t s, int phase) {
  bf_filter* f = const_cast<bf_filter*>(fc);
  PhaseMark m;
  if (!f->timing) return m;
  m.a = pool_event(f);
  if (m.a && cudaEventRecord(m.a, s) == cudaSuccess) m.phase = phase;
  return m;
}

void phase_end(const bf_filter* fc, cudaStream_t s, const PhaseMark& m, uint32_t launches) {
  bf_filter* f = const_cast<bf_filter*>(fc);
  if (m.phase < 0) return;
  cudaEvent_t b = pool_event(f);
  if (b && cudaEventRecord(b, s) == cudaSuccess) f->segs.push_back({m.phase, m.a, b, launches});
}

// a new call: count its launches from zero (timing marks accumulate until read)
void begin_call(const bf_filter* fc) { const_cast<bf_filter*>(fc)->last_launches = 0; }

bf_status launch_sbf(const bf_filter* f, int op, const uint64_t* keys, uint64_t n, uint8_t* out,
                     cudaStream_t stream) {
  if (reinterpret_cast<uintptr_t>(keys) % 8 || (op == BF_OP_CONTAINS && !out))
    return fail(BF_EINVAL, "keys must be 8-byte aligned and out non-NULL");
  const bf_layout& l = f->layout[op];
  const KernelEntry* e = f->entry[op];
  uint32_t grid = 0;
  bf_status s = resolve_grid(e->fn, f->device, l.block_threads, l.grid_ctas, n, l.kpt, &grid);
  if (s != BF_OK) return s;
  SbfArgs a{f->words, f->p.num_blocks, keys, n, out, f->p.seed + 0x27D4EB2F165667C5ull + 8ull, l.flags,
            f->p.num_blocks < (1ull << 32) ? 0 : (f->p.num_blocks == (1ull << 32) ? 1 : 2)};
  void* args[] = {&a};
  const PhaseMark pm = phase_begin(f, stream, op == BF_OP_ADD ? BF_PHASE_ADD_DIRECT : BF_PHASE_CONTAINS_DIRECT);
  cudaError_t err = cudaLaunchKernel(e->fn, dim3(grid), dim3(l.block_threads), args, 0, stream);
  if (err != cudaSuccess) return cuda_fail(err, op == BF_OP_ADD ? "launch add kernel" : "launch contains kernel");
  phase_end(f, stream, pm, 1);
  const_cast<bf_filter*>(f)->last_launches += 1;
  return BF_OK;
}

// --- L2-blocked construction ------------------------------------------------

struct PartPlan {
  uint32_t shift = 0, nparts = 0;
};

// slice geometry: 2^shift blocks per slice, at most static_cast<uint32_t>(kMaxParts) slices
PartPlan part_plan(const bf_filter* f) {
  PartPlan pl;
  const uint64_t b = f->p.num_blocks;
  const uint32_t block_log2 = static_cast<uint32_t>(__builtin_ctz(f->p.block_bits / 8));
  uint32_t shift = f->part.slice_log2 > block_log2 ? f->part.slice_log2 - block_log2 : 0;
  while (((b + (1ull << shift) - 1) >> shift) > static_cast<uint32_t>(kMaxParts)) ++shift;
  pl.shift = shift;
  pl.nparts = static_cast<uint32_t>((b + (1ull << shift) - 1) >> shift);
  return pl;
}

// slots per slice buffer for a pass of `keys` keys: the expected count of the
// fullest slice plus 8 standard deviations, rounded up to the record tile
uint64_t part_cap(const bf_filter* f, const PartPlan& pl, uint64_t keys) {
  if (f->part.cap_override) return f->part.cap_override;
  const double frac = std::min(1.0, static_cast<double>(1ull << pl.shift) / static_cast<double>(f->p.num_blocks));
  const double mean = static_cast<double>(keys) * frac;
  const double cap = mean + 8.0 * std::sqrt(mean) + 256.0;
  return (static_cast<uint64_t>(cap) + kRecTile - 1) / kRecTile * kRecTile;
}

bool use_partitioned(const bf_filter* f, uint64_t n) {
  if (f->part.mode == BF_PART_OFF || f->p.num_blocks > (1ull << 32) || csbf_groups(f->p)) return false;
  const PartPlan pl = part_plan(f);
  if (pl.nparts < 2) return false;
  if (f->part.mode == BF_PART_ON) return true;
  return f->nbytes * 2 > f->l2_bytes && n >= f->p.num_blocks / 2;
}

const KernelEntry* find_op(int op, const bf_params& p, uint32_t cg, uint32_t phi, uint32_t kpt) {
  bf_layout l{};
  l.cg = cg;
  l.phi = phi;
  l.kpt = kpt;
  return find_sbf(op, p, l);
}

bf_status ensure_ws(void** ws, uint64_t* ws_bytes, uint64_t bytes) {
  if (*ws && *ws_bytes >= bytes) return BF_OK;
  if (*ws) {
    cudaFree(*ws);
    *ws = nullptr;
    *ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ws = nullptr;
    return fail(BF_ENOMEM, "partition workspace allocation failed");
  }
  *ws_bytes = bytes;
  return BF_OK;
}

bf_status ensure_part_ws(bf_filter* f, uint64_t bytes) { return ensure_ws(&f->part_ws, &f->part_ws_bytes, bytes); }

// the status word the slice-partitioned kernels report failed index checks in
bf_status ensure_status(bf_filter* f) {
  if (f->status) return BF_OK;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(BF_ENOMEM, "status word allocation failed");
  }
  if ((e = cudaMemset(p, 0, 256)) != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(e, "cudaMemset");
  }
  f->status = static_cast<uint32_t*>(p);
  return BF_OK;
}

// Kernels and launch shapes of a slice-partitioned construction.
struct PartLaunch {
  const KernelEntry* pe = nullptr;  // slice partition
  const KernelEntry* re = nullptr;  // record insert (the add layout)
  size_t smem = 0;
  uint32_t max_grid = 0;    // partition CTAs: SMs x min(resident, max_per_sm)
  uint32_t per_launch = 1;  // slices per record-insert launch (one window)
};

// Shared-memory carveout of the kernels that share SMs with the slice
// partition: kBesidePartitionCarveout in the overlapped and SM-staged
// schedules (an SM that one of them brought up with a large L1, the default
// without shared memory, would take no partition CTA until it went idle),
// the default elsewhere (the record probes run faster with the whole L1).
bf_status set_carveout(const void* fn, int carveout) {
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
  return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaFuncSetAttribute(carveout)");
}

bf_status prepare_part_launch(bf_filter* f, const PartPlan& pl, int max_per_sm, bool beside, PartLaunch* L) {
  bf_status st = ensure_status(f);
  if (st != BF_OK) return st;
  const bf_layout& l = f->layout[BF_OP_ADD];
  L->pe = find_op(3, f->p, 0, 0, 0);
  L->re = find_op(2, f->p, l.cg, l.phi, l.kpt);
  if (!L->pe || !L->re) return fail(BF_EUNSUPPORTED, "no partition kernels for this geometry");
  if ((st = set_carveout(L->re->fn, beside ? kBesidePartitionCarveout : cudaSharedmemCarveoutDefault)) != BF_OK)
    return st;
  L->smem = partition_smem_bytes(static_cast<int>(pl.nparts));
  cudaError_t e =
      cudaFuncSetAttribute(L->pe->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L->smem));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(partition)");
  int sms = 0, per_sm = 0;
  bf_status s = sm_count(f->device, &sms);
  if (s != BF_OK) return s;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L->pe->fn, kPartThreads, L->smem)) != cudaSuccess)
    return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(partition)");
  L->max_grid = static_cast<uint32_t>(sms * std::max(1, std::min(per_sm, max_per_sm)));
  const uint32_t slice_bytes_log2 = pl.shift + static_cast<uint32_t>(__builtin_ctz(f->p.block_bits / 8));
  L->per_launch = f->part.window_log2 > slice_bytes_log2
                      ? 1u << std::min<uint32_t>(f->part.window_log2 - slice_bytes_log2, 20)
                      : 1u;
  return BF_OK;
}

// Zero the slice counts and partition keys[0, cnt) into the slice buffers.
bf_status launch_partition_pass(bf_filter* f, const PartLaunch& L, const PartPlan& pl, const uint64_t* keys,
                                uint64_t cnt, uint64_t cap, unsigned long long* counts, uint64_t* records,
                                cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counts, 0, 8ull * pl.nparts, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  PartArgs pa{keys, cnt, f->p.seed + 0x27D4EB2F165667C5ull + 8ull, f->p.num_blocks,
              f->p.num_blocks < (1ull << 32) ? 0 : 1, pl.shift, pl.nparts, cap, counts, records, f->words,
              nullptr, nullptr, f->status};
  const uint64_t tiles = (cnt + part_tile(false) - 1) / part_tile(false);
  const uint32_t grid = static_cast<uint32_t>(std::min<uint64_t>(tiles, L.max_grid));
  void* pargs[] = {&pa};
  const PhaseMark pm = phase_begin(f, stream, BF_PHASE_PARTITION_ADD);
  if ((e = cudaLaunchKernel(L.pe->fn, dim3(grid), dim3(kPartThreads), pargs, L.smem, stream)) != cudaSuccess)
    return cuda_fail(e, "launch partition kernel");
  phase_end(f, stream, pm, 1);
  f->last_launches += 1;
  return BF_OK;
}

// Insert the slice buffers' records, one window of slices per launch.
bf_status launch_record_windows(bf_filter* f, const PartLaunch& L, const PartPlan& pl, const uint64_t* records,
                                const unsigned long long* counts, uint64_t cap, cudaStream_t stream) {
  const bf_layout& l = f->layout[BF_OP_ADD];
  const PhaseMark pm = phase_begin(f, stream, BF_PHASE_RECORD_INSERT);
  uint32_t nl = 0;
  for (uint32_t plo = 0; plo < pl.nparts; plo += L.per_launch, ++nl) {
    const uint32_t phi = std::min(pl.nparts, plo + L.per_launch);
    RecArgs ra{f->words, records, counts, plo, phi, cap, l.flags, f->p.num_blocks, f->status};
    uint32_t rgrid = 0;
    bf_status s = resolve_grid(L.re->fn, f->device, l.block_threads, l.grid_ctas, (phi - plo) * cap, l.kpt, &rgrid);
    if (s != BF_OK) return s;
    void* rargs[] = {&ra};
    cudaError_t e = cudaLaunchKernel(L.re->fn, dim3(rgrid), dim3(l.block_threads), rargs, 0, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch record-insert kernel");
    f->last_launches += 1;
  }
  phase_end(f, stream, pm, nl);
  return BF_OK;
}

// One partition pass over all keys per chunk_keys, then its record inserts.
bf_status launch_partitioned_serial(bf_filter* f, const uint64_t* keys, uint64_t n, cudaStream_t stream) {
  const PartPlan pl = part_plan(f);
  const uint64_t pass = std::min<uint64_t>(n, f->part.chunk_keys);
  const uint64_t cap_max = part_cap(f, pl, pass);
  const uint64_t counts_bytes = 8ull * static_cast<uint32_t>(kMaxParts);
  bf_status s = ensure_part_ws(f, counts_bytes + static_cast<uint64_t>(pl.nparts) * cap_max * 8);
  if (s != BF_OK) return launch_sbf(f, BF_OP_ADD, keys, n, nullptr, stream);  // no memory: direct kernel
  PartLaunch L;
  if ((s = prepare_part_launch(f, pl, f->part.part_ctas ? static_cast<int>(f->part.part_ctas) : 1 << 30, false,
                                &L)) !=
      BF_OK)
    return s;
  unsigned long long* counts = static_cast<unsigned long long*>(f->part_ws);
  uint64_t* records = reinterpret_cast<uint64_t*>(static_cast<char*>(f->part_ws) + counts_bytes);
  for (uint64_t lo = 0; lo < n; lo += pass) {
    const uint64_t cnt = std::min(pass, n - lo);
    const uint64_t cap = part_cap(f, pl, cnt);
    if ((s = launch_partition_pass(f, L, pl, keys + lo, cnt, cap, counts, records, stream)) != BF_OK) return s;
    if ((s = launch_record_windows(f, L, pl, records, counts, cap, stream)) != BF_OK) return s;
  }
  return BF_OK;
}

// Construction in at least `passes` passes over two alternating workspaces,
// overlapping the two phases: the record inserts of pass i (bound by the
// SM-to-L2 atomic path, little DRAM traffic) run on the filter's second
// stream while the partition of pass i + 1 (a DRAM stream) runs on `stream`,
// its grid limited to part_ctas CTAs per SM so that record-insert CTAs find
// room beside it.  Ordering: pass i + 2 reuses pass i's workspace only after
// pass i's record inserts (event), and the caller's stream waits for every
// record insert.  Without room for two workspaces it falls back to the
// serial schedule.
bf_status launch_partitioned_overlap(bf_filter* f, const uint64_t* keys, uint64_t n, cudaStream_t stream,
                                     uint64_t passes, int part_ctas) {
  const PartPlan pl = part_plan(f);
  const uint64_t pass = std::min<uint64_t>(f->part.chunk_keys, (n + passes - 1) / passes);
  const uint64_t counts_bytes = 8ull * static_cast<uint32_t>(kMaxParts);
  const uint64_t ws_one = counts_bytes + static_cast<uint64_t>(pl.nparts) * part_cap(f, pl, pass) * 8;
  if (ensure_part_ws(f, 2 * ws_one) != BF_OK) return launch_partitioned_serial(f, keys, n, stream);
  cudaError_t e;
  if (!f->rec_stream && (e = cudaStreamCreateWithFlags(&f->rec_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  for (int i = 0; i < 2; ++i) {
    if (!f->ev_part[i] && (e = cudaEventCreateWithFlags(&f->ev_part[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    if (!f->ev_rec[i] && (e = cudaEventCreateWithFlags(&f->ev_rec[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
  }
  PartLaunch L;
  bf_status s = prepare_part_launch(f, pl, part_ctas, true, &L);
  if (s != BF_OK) return s;
  bool used[2] = {false, false};
  uint64_t i = 0;
  for (uint64_t lo = 0; lo < n; lo += pass, ++i) {
    const int w = static_cast<int>(i & 1);
    const uint64_t cnt = std::min(pass, n - lo);
    const uint64_t cap = part_cap(f, pl, cnt);
    char* base = static_cast<char*>(f->part_ws) + w * ws_one;
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(base);
    uint64_t* records = reinterpret_cast<uint64_t*>(base + counts_bytes);
    if (used[w] && (e = cudaStreamWaitEvent(stream, f->ev_rec[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if ((s = launch_partition_pass(f, L, pl, keys + lo, cnt, cap, counts, records, stream)) != BF_OK) return s;
    if ((e = cudaEventRecord(f->ev_part[w], stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(f->rec_stream, f->ev_part[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if ((s = launch_record_windows(f, L, pl, records, counts, cap, f->rec_stream)) != BF_OK) return s;
    if ((e = cudaEventRecord(f->ev_rec[w], f->rec_stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    used[w] = true;
  }
  for (int w = 0; w < 2; ++w)
    if (used[w] && (e = cudaStreamWaitEvent(stream, f->ev_rec[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
  return BF_OK;
}

bf_status launch_partitioned(bf_filter* f, const uint64_t* keys, uint64_t n, cudaStream_t stream) {
  if (f->part.passes >= 2 && n >= 2ull * part_tile(false))
    return launch_partitioned_overlap(f, keys, n, stream, f->part.passes,
                                      f->part.part_ctas ? static_cast<int>(f->part.part_ctas) : 1 << 30);
  return launch_partitioned_serial(f, keys, n, stream);
}

// Construction from keys the kernels read in host memory: the slice
// partition is bound by the host link, the record inserts (L2, no host
// traffic) are not, so the overlapped schedule runs with at least
// max(kHostPasses, passes) passes and part_ctas (default kHostPartCtas)
// partition CTAs per SM (enough for the link).
constexpr uint64_t kHostPasses = 8;
constexpr int kHostPartCtas = 1;
// Partition CTAs per SM beside the staging kernel's CTA (its 4096 registers
// leave room for three partition CTAs of either kind).
constexpr int kStagedPartCtas = 3;

// Keys per pass of a staged host-buffer call: n split into passes - 3/4
// equal shares, so the last pass is about a quarter of the others (only the
// last pass's device work is not hidden behind the staging of the next one),
// rounded up to 256 keys (keeps every pass 16-byte aligned when the buffer
// is), at most `cap`.
uint64_t host_pass_keys(uint64_t n, uint64_t passes, uint64_t cap) {
  const uint64_t share = (4 * n + 4 * passes - 4) / (4 * passes - 3);  // ceil(4n / (4 passes - 3))
  return std::min<uint64_t>(cap, (share + 255) / 256 * 256);
}

int host_part_ctas(const bf_filter* f) { return f->part.part_ctas ? static_cast<int>(f->part.part_ctas) : kHostPartCtas; }

bf_status launch_partitioned_host(bf_filter* f, const uint64_t* keys, uint64_t n, cudaStream_t stream) {
  return launch_partitioned_overlap(f, keys, n, stream, std::max<uint64_t>(kHostPasses, f->part.passes),
                                    host_part_ctas(f));
}

bool use_partitioned_lookup(const bf_filter* f, uint64_t n) {
  if (f->part.lookup_mode == BF_PART_OFF || f->p.num_blocks > (1ull << 32) || csbf_groups(f->p)) return false;
  const PartPlan pl = part_plan(f);
  if (pl.nparts < 2) return false;
  if (f->part.lookup_mode == BF_PART_ON) return true;
  return f->nbytes * 2 > f->l2_bytes && n >= f->p.num_blocks / 4;
}

const KernelEntry* find_expand() {
  for (const auto& e : registry().sbf)
    if (e.op == 6) return &e;
  return nullptr;
}

// Kernels, launch shapes and workspace layout of a slice-partitioned lookup.
struct LookupLaunch {
  const KernelEntry* pe = nullptr;  // slice partition (lookup)
  const KernelEntry* qe = nullptr;  // record probe (the lookup layout)
  const KernelEntry* xe = nullptr;  // bitmap expansion
  size_t smem = 0;
  uint32_t part_grid = 0;    // partition CTAs: SMs x min(resident, max_per_sm)
  uint32_t per_launch = 1;   // slices per record-probe launch (one window)
  uint32_t xgrid_cap = 0;    // expansion CTAs: at most SMs x 8
  uint64_t ws_bytes = 0;     // one pass's workspace: counts | records | indexes | bitmap
  uint64_t rec_off = 0, idx_off = 0, bitmap_off = 0;
};

bf_status prepare_lookup(bf_filter* f, const PartPlan& pl, uint64_t pass, int max_per_sm, bool beside,
                         LookupLaunch* L) {
  const uint64_t cap_max = part_cap(f, pl, pass);
  const uint64_t counts_bytes = 8ull * kMaxParts;
  const uint64_t rec_bytes = static_cast<uint64_t>(pl.nparts) * cap_max * 8;
  const uint64_t idx_bytes = static_cast<uint64_t>(pl.nparts) * cap_max * 4;
  const uint64_t bitmap_bytes = ((pass + 31) / 32 * 4 + 255) / 256 * 256;
  L->rec_off = counts_bytes;
  L->idx_off = counts_bytes + rec_bytes;
  L->bitmap_off = counts_bytes + rec_bytes + idx_bytes;
  L->ws_bytes = L->bitmap_off + bitmap_bytes;
  L->pe = find_op(5, f->p, 0, 0, 0);
  const bf_layout& l = f->layout[BF_OP_CONTAINS];
  L->qe = find_op(4, f->p, l.cg, l.phi, l.kpt);
  L->xe = find_expand();
  if (!L->pe || !L->qe || !L->xe) return fail(BF_EUNSUPPORTED, "no partitioned lookup kernels for this geometry");
  bf_status s = ensure_status(f);
  if (s != BF_OK) return s;
  const int carveout = beside ? kBesidePartitionCarveout : cudaSharedmemCarveoutDefault;
  if ((s = set_carveout(L->qe->fn, carveout)) != BF_OK || (s = set_carveout(L->xe->fn, carveout)) != BF_OK) return s;
  L->smem = partition_smem_bytes(static_cast<int>(pl.nparts), true);
  cudaError_t e =
      cudaFuncSetAttribute(L->pe->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L->smem));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(partition)");
  int sms = 0, per_sm = 0;
  if ((s = sm_count(f->device, &sms)) != BF_OK) return s;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L->pe->fn, kPartThreads, L->smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(partition)");
  L->part_grid = static_cast<uint32_t>(sms * std::max(1, std::min(per_sm, max_per_sm)));
  L->xgrid_cap = static_cast<uint32_t>(sms) * 8;
  const uint32_t slice_bytes_log2 = pl.shift + static_cast<uint32_t>(__builtin_ctz(f->p.block_bits / 8));
  L->per_launch = f->part.window_log2 > slice_bytes_log2
                      ? 1u << std::min<uint32_t>(f->part.window_log2 - slice_bytes_log2, 20)
                      : 1u;
  return BF_OK;
}

// One lookup pass over queries keys[0, cnt) with the workspace at `ws`: the
// partition on `part_stream`, then the record probes and the bitmap
// expansion into out[0, cnt) on `probe_stream`.  `ev` (required when the two
// streams differ, else optional) is recorded on `part_stream` once the
// partition has read the queries; `probe_stream` waits for it.
bf_status launch_lookup_pass(bf_filter* f, const LookupLaunch& L, const PartPlan& pl, const uint64_t* keys,
                             uint64_t cnt, uint8_t* out, char* ws, cudaStream_t part_stream,
                             cudaStream_t probe_stream, cudaEvent_t ev) {
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(ws);
  uint64_t* records = reinterpret_cast<uint64_t*>(ws + L.rec_off);
  uint32_t* idx = reinterpret_cast<uint32_t*>(ws + L.idx_off);
  uint32_t* bitmap = reinterpret_cast<uint32_t*>(ws + L.bitmap_off);
  const uint64_t cap = part_cap(f, pl, cnt);
  const bf_layout& l = f->layout[BF_OP_CONTAINS];
  cudaError_t e;
  if ((e = cudaMemsetAsync(counts, 0, 8ull * pl.nparts, part_stream)) != cudaSuccess)
    return cuda_fail(e, "cudaMemsetAsync");
  if ((e = cudaMemsetAsync(bitmap, 0, (cnt + 31) / 32 * 4, part_stream)) != cudaSuccess)
    return cuda_fail(e, "cudaMemsetAsync");
  PartArgs pa{keys, cnt, f->p.seed + 0x27D4EB2F165667C5ull + 8ull, f->p.num_blocks,
              f->p.num_blocks < (1ull << 32) ? 0 : 1, pl.shift, pl.nparts, cap, counts, records, f->words, idx,
              bitmap, f->status};
  const uint64_t tiles = (cnt + part_tile(true) - 1) / part_tile(true);
  const uint32_t grid = static_cast<uint32_t>(std::min<uint64_t>(tiles, L.part_grid));
  void* pargs[] = {&pa};
  PhaseMark pm = phase_begin(f, part_stream, BF_PHASE_PARTITION_LOOKUP);
  if ((e = cudaLaunchKernel(L.pe->fn, dim3(grid), dim3(kPartThreads), pargs, L.smem, part_stream)) != cudaSuccess)
    return cuda_fail(e, "launch partition kernel (lookup)");
  phase_end(f, part_stream, pm, 1);
  f->last_launches += 1;
  if (ev && (e = cudaEventRecord(ev, part_stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if (probe_stream != part_stream && (e = cudaStreamWaitEvent(probe_stream, ev, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamWaitEvent");
  pm = phase_begin(f, probe_stream, BF_PHASE_RECORD_PROBE);
  uint32_t nl = 0;
  for (uint32_t plo = 0; plo < pl.nparts; plo += L.per_launch, ++nl) {
    const uint32_t phi = std::min(pl.nparts, plo + L.per_launch);
    ProbeArgs qa{f->words, records, idx, counts, plo, phi, cap, bitmap, l.flags, f->p.num_blocks, f->status};
    uint32_t qgrid = 0;
    bf_status s = resolve_grid(L.qe->fn, f->device, l.block_threads, l.grid_ctas, (phi - plo) * cap, l.kpt, &qgrid);
    if (s != BF_OK) return s;
    void* qargs[] = {&qa};
    if ((e = cudaLaunchKernel(L.qe->fn, dim3(qgrid), dim3(l.block_threads), qargs, 0, probe_stream)) != cudaSuccess)
      return cuda_fail(e, "launch record-probe kernel");
    f->last_launches += 1;
  }
  phase_end(f, probe_stream, pm, nl);
  ExpandArgs xa{bitmap, cnt, out};
  const uint64_t words = (cnt + 31) / 32;
  const uint32_t xgrid = static_cast<uint32_t>(std::min<uint64_t>((words + 255) / 256, L.xgrid_cap));
  void* xargs[] = {&xa};
  pm = phase_begin(f, probe_stream, BF_PHASE_BITMAP_EXPAND);
  if ((e = cudaLaunchKernel(L.xe->fn, dim3(xgrid), dim3(256), xargs, 0, probe_stream)) != cudaSuccess)
    return cuda_fail(e, "launch bitmap expansion");
  phase_end(f, probe_stream, pm, 1);
  f->last_launches += 1;
  return BF_OK;
}

// Slice-partitioned lookup: per pass of at most lookup_chunk_keys queries,
// partition the queries by slice (with their indices), probe each L2-sized
// window's records, setting a bit per positive query in a result bitmap
// that stays in L2, then expand the bitmap into the result bytes.
bf_status launch_contains_partitioned(const bf_filter* fc, const uint64_t* keys, uint64_t n, uint8_t* out,
                                      cudaStream_t stream) {
  bf_filter* f = const_cast<bf_filter*>(fc);
  const PartPlan pl = part_plan(f);
  const uint64_t pass = std::min<uint64_t>(n, f->part.lookup_chunk_keys);
  LookupLaunch L;
  bf_status s = prepare_lookup(f, pl, pass, 1 << 30, false, &L);
  if (s != BF_OK) return s;
  if (ensure_ws(&f->look_ws, &f->look_ws_bytes, L.ws_bytes) != BF_OK)
    return launch_sbf(f, BF_OP_CONTAINS, keys, n, out, stream);  // no memory: direct kernel
  for (uint64_t lo = 0; lo < n; lo += pass) {
    const uint64_t cnt = std::min(pass, n - lo);
    if ((s = launch_lookup_pass(f, L, pl, keys + lo, cnt, out + lo, static_cast<char*>(f->look_ws), stream, stream,
                                nullptr)) != BF_OK)
      return s;
  }
  return BF_OK;
}

// Lookup of queries the kernels read in host memory (results written there):
// the partition reads the host link, the probes do not.  At least
// kHostPasses passes over two alternating workspaces; the probes and the
// expansion of pass i run on the filter's second stream while the partition
// of pass i + 1 (kHostPartCtas CTAs per SM) reads the next queries.
bf_status launch_contains_partitioned_host(bf_filter* f, const uint64_t* keys, uint64_t n, uint8_t* out,
                                           cudaStream_t stream) {
  const PartPlan pl = part_plan(f);
  const uint64_t passes = std::max<uint64_t>(kHostPasses, f->part.passes);
  const uint64_t pass = std::min<uint64_t>(f->part.lookup_chunk_keys, (n + passes - 1) / passes);
  LookupLaunch L;
  bf_status s = prepare_lookup(f, pl, pass, host_part_ctas(f), true, &L);
  if (s != BF_OK) return s;
  if (ensure_ws(&f->look_ws, &f->look_ws_bytes, 2 * L.ws_bytes) != BF_OK)
    return launch_contains_partitioned(f, keys, n, out, stream);
  cudaError_t e;
  if (!f->rec_stream && (e = cudaStreamCreateWithFlags(&f->rec_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  for (int i = 0; i < 2; ++i) {
    if (!f->ev_part[i] && (e = cudaEventCreateWithFlags(&f->ev_part[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    if (!f->ev_rec[i] && (e = cudaEventCreateWithFlags(&f->ev_rec[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
  }
  bool used[2] = {false, false};
  uint64_t i = 0;
  for (uint64_t lo = 0; lo < n; lo += pass, ++i) {
    const int w = static_cast<int>(i & 1);
    const uint64_t cnt = std::min(pass, n - lo);
    if (used[w] && (e = cudaStreamWaitEvent(stream, f->ev_rec[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    char* ws = static_cast<char*>(f->look_ws) + w * L.ws_bytes;
    if ((s = launch_lookup_pass(f, L, pl, keys + lo, cnt, out + lo, ws, stream, f->rec_stream, f->ev_part[w])) !=
        BF_OK)
      return s;
    if ((e = cudaEventRecord(f->ev_rec[w], f->rec_stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    used[w] = true;
  }
  for (int w = 0; w < 2; ++w)
    if (used[w] && (e = cudaStreamWaitEvent(stream, f->ev_rec[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
  return BF_OK;
}

bf_status run_contains(const bf_filter* f, const uint64_t* keys, uint64_t n, uint8_t* out, cudaStream_t stream) {
  if (use_partitioned_lookup(f, n)) return launch_contains_partitioned(f, keys, n, out, stream);
  return launch_sbf(f, BF_OP_CONTAINS, keys, n, out, stream);
}

bf_status run_add(bf_filter* f, const uint64_t* keys, uint64_t n, cudaStream_t stream) {
  if (use_partitioned(f, n)) return launch_partitioned(f, keys, n, stream);
  return launch_sbf(f, BF_OP_ADD, keys, n, nullptr, stream);
}

// Can the kernels read (and for results, write) this host buffer directly?
bool device_can_access(const bf_filter* f, const void* h) {
  if (f->host_access == BF_HOST_STAGED) return false;
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, h) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) return true;
  if (attr.type == cudaMemoryTypeHost) return attr.devicePointer == h;
  int pageable = 0;
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, f->device);
  return pageable == 1;
}

// Bytes of one staging slot: the keys, then the results, each region padded
// to 256 bytes so every slot's key pointer keeps the alignment the kernels'
// vector loads need.
uint64_t keys_region(uint64_t chunk_keys) { return (chunk_keys * 8 + 255) / 256 * 256; }
uint64_t slot_bytes(uint64_t chunk_keys) { return keys_region(chunk_keys) + (chunk_keys + 255) / 256 * 256; }

bf_status ensure_pipeline(bf_filter* f) {
  if (f->staging) return BF_OK;
  const uint64_t per = slot_bytes(f->chunk_keys);
  cudaError_t e = cudaMalloc(&f->staging, per * kPipelineDepth);
  if (e != cudaSuccess) {
    cudaGetLastError();
    f->staging = nullptr;
    return fail(BF_ENOMEM, "staging allocation failed");
  }
  for (int i = 0; i < kPipelineDepth; ++i) {
    if (!f->pipe[i] && (e = cudaStreamCreateWithFlags(&f->pipe[i], cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    if (!f->ev_done[i] && (e = cudaEventCreateWithFlags(&f->ev_done[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
  }
  if (!f->ev_start && (e = cudaEventCreateWithFlags(&f->ev_start, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  return BF_OK;
}

void release_pipeline(bf_filter* f) {
  if (f->staging) cudaFree(f->staging);
  f->staging = nullptr;
  if (f->rec_stream) cudaStreamDestroy(f->rec_stream);
  f->rec_stream = nullptr;
  for (int i = 0; i < 2; ++i) {
    if (f->ev_part[i]) cudaEventDestroy(f->ev_part[i]);
    if (f->ev_rec[i]) cudaEventDestroy(f->ev_rec[i]);
    f->ev_part[i] = f->ev_rec[i] = nullptr;
  }
  for (int i = 0; i < kPipelineDepth; ++i) {
    if (f->pipe[i]) cudaStreamDestroy(f->pipe[i]);
    if (f->ev_done[i]) cudaEventDestroy(f->ev_done[i]);
    f->pipe[i] = nullptr;
    f->ev_done[i] = nullptr;
  }
  if (f->ev_start) cudaEventDestroy(f->ev_start);
  f->ev_start = nullptr;
  if (f->hstage) cudaFree(f->hstage);
  f->hstage = nullptr;
  f->hstage_bytes = 0;
  for (cudaStream_t* st : {&f->h2d, &f->d2h}) {
    if (*st) cudaStreamDestroy(*st);
    *st = nullptr;
  }
  for (int i = 0; i < 2; ++i)
    for (cudaEvent_t* ev : {&f->ev_copied[i], &f->ev_consumed[i], &f->ev_computed[i], &f->ev_drained[i]}) {
      if (*ev) cudaEventDestroy(*ev);
      *ev = nullptr;
    }
}

// Is this host buffer page-locked (cudaHostAlloc / cudaHostRegister)?  The
// copy engine then copies to it asynchronously.
bool is_page_locked(const void* h) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, h) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeHost;
}

bf_status ensure_stream(cudaStream_t* st) {
  cudaError_t e;
  if (!*st && (e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  return BF_OK;
}

bf_status ensure_event(cudaEvent_t* ev) {
  cudaError_t e;
  if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  return BF_OK;
}

bf_status ensure_copy_streams(bf_filter* f) {
  bf_status s;
  if (!f->h2d) {
    // highest priority: the staging kernel's CTAs take the first free slots
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&f->h2d, cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithPriority");
  }
  if ((s = ensure_stream(&f->d2h)) != BF_OK) return s;
  if ((s = ensure_event(&f->ev_start)) != BF_OK) return s;
  for (int i = 0; i < 2; ++i)
    if ((s = ensure_event(&f->ev_copied[i])) != BF_OK || (s = ensure_event(&f->ev_consumed[i])) != BF_OK ||
        (s = ensure_event(&f->ev_computed[i])) != BF_OK || (s = ensure_event(&f->ev_drained[i])) != BF_OK)
      return s;
  return BF_OK;
}

// Start the copy streams after the work already on `stream`.
bf_status fork_copies(bf_filter* f, cudaStream_t stream) {
  cudaError_t e;
  if ((e = cudaEventRecord(f->ev_start, stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if ((e = cudaStreamWaitEvent(f->h2d, f->ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(f->d2h, f->ev_start, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamWaitEvent");
  return BF_OK;
}

// Copy n host keys into device memory on the copy-in stream: the staging
// kernel (one CTA per SM) or the copy engine.
bf_status stage_keys(bf_filter* f, const uint64_t* h, uint64_t* d, uint64_t n, int sms, bool sm_copy) {
  uint32_t launches = 0;
  const PhaseMark pm = phase_begin(f, f->h2d, BF_PHASE_HOST_STAGE);
  cudaError_t e = sm_copy ? launch_host_stage(h, d, n, static_cast<uint32_t>(sms), f->h2d, &launches)
                          : cudaMemcpyAsync(d, h, n * 8, cudaMemcpyHostToDevice, f->h2d);
  if (e != cudaSuccess) return cuda_fail(e, sm_copy ? "launch staging kernel" : "cudaMemcpyAsync H2D");
  phase_end(f, f->h2d, pm, launches);
  f->last_launches += launches;
  return BF_OK;
}

// Construction from host keys in passes staged through device memory: on
// the copy-in stream (highest priority) each pass's keys are copied into one
// of two device staging slots, by the staging kernel on one CTA slot per SM
// when the kernels can address the keys (sm_copy), else by the copy engine,
// while `stream` partitions (kStagedPartCtas CTAs per SM beside the staging
// kernel) and inserts the previous pass from device memory; a pass's device
// work takes a fraction of its copy, so the call costs about the copy of all
// keys plus the device work of the last pass.  Pass i + 2 refills pass i's
// slot once pass i's partition has read it.  Returns BF_ENOMEM, having
// queued nothing, when the workspaces do not fit.
bf_status launch_partitioned_staged(bf_filter* f, const uint64_t* h_keys, uint64_t n, cudaStream_t stream,
                                    bool sm_copy) {
  const PartPlan pl = part_plan(f);
  const uint64_t pass = host_pass_keys(n, std::max<uint64_t>(kHostPasses, f->part.passes), f->part.chunk_keys);
  const uint64_t counts_bytes = 8ull * static_cast<uint32_t>(kMaxParts);
  const uint64_t kbytes = (pass * 8 + 255) / 256 * 256;
  if (ensure_part_ws(f, counts_bytes + static_cast<uint64_t>(pl.nparts) * part_cap(f, pl, pass) * 8) != BF_OK ||
      ensure_ws(&f->hstage, &f->hstage_bytes, 2 * kbytes) != BF_OK)
    return BF_ENOMEM;
  bf_status s = ensure_copy_streams(f);
  if (s != BF_OK) return s;
  PartLaunch L;
  if ((s = prepare_part_launch(f, pl, sm_copy ? kStagedPartCtas : 1 << 30, sm_copy, &L)) != BF_OK) return s;
  int sms = 0;
  if ((s = sm_count(f->device, &sms)) != BF_OK) return s;
  if ((s = fork_copies(f, stream)) != BF_OK) return s;
  unsigned long long* counts = static_cast<unsigned long long*>(f->part_ws);
  uint64_t* records = reinterpret_cast<uint64_t*>(static_cast<char*>(f->part_ws) + counts_bytes);
  cudaError_t e;
  uint64_t i = 0;
  for (uint64_t lo = 0; lo < n; lo += pass, ++i) {
    const int w = static_cast<int>(i & 1);
    const uint64_t cnt = std::min(pass, n - lo);
    uint64_t* d_keys = reinterpret_cast<uint64_t*>(static_cast<char*>(f->hstage) + w * kbytes);
    if (i >= 2 && (e = cudaStreamWaitEvent(f->h2d, f->ev_consumed[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if ((s = stage_keys(f, h_keys + lo, d_keys, cnt, sms, sm_copy)) != BF_OK) return s;
    if ((e = cudaEventRecord(f->ev_copied[w], f->h2d)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(stream, f->ev_copied[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    const uint64_t cap = part_cap(f, pl, cnt);
    if ((s = launch_partition_pass(f, L, pl, d_keys, cnt, cap, counts, records, stream)) != BF_OK) return s;
    if ((e = cudaEventRecord(f->ev_consumed[w], stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((s = launch_record_windows(f, L, pl, records, counts, cap, stream)) != BF_OK) return s;
  }
  return BF_OK;
}

// Lookup of host queries in passes staged through device memory: pass i's
// queries are copied into a staging slot on the copy-in stream (the staging
// kernel when the kernels can address the buffers, else the copy engine),
// and the pass runs on `stream` (partition, probes, expansion into the
// slot's result bytes); the copy engine takes the results back on the
// copy-out stream, so both directions of the link stay busy while the device
// works.  For a pageable h_out the kernels can address (results_in_place),
// whose copy would wait for the results before returning, the expansion
// writes into h_out itself (slower: about 80 GB/s of byte stores over the
// link, on `stream`).  Pass i + 2 refills slot i % 2 once pass i's partition
// has read its queries, and overwrites its results once they have reached
// the host.
// Returns BF_ENOMEM, having queued nothing, when the workspaces do not fit.
bf_status launch_contains_partitioned_staged(bf_filter* f, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                                             cudaStream_t stream, bool sm_copy, bool results_in_place) {
  const PartPlan pl = part_plan(f);
  const uint64_t pass =
      host_pass_keys(n, std::max<uint64_t>(kHostPasses, f->part.passes), f->part.lookup_chunk_keys);
  LookupLaunch L;
  bf_status s = prepare_lookup(f, pl, pass, sm_copy ? kStagedPartCtas : 1 << 30, sm_copy, &L);
  if (s != BF_OK) return s;
  const uint64_t kbytes = (pass * 8 + 255) / 256 * 256;
  const uint64_t slot = kbytes + (results_in_place ? 0 : (pass + 255) / 256 * 256);
  if (ensure_ws(&f->look_ws, &f->look_ws_bytes, L.ws_bytes) != BF_OK ||
      ensure_ws(&f->hstage, &f->hstage_bytes, 2 * slot) != BF_OK)
    return BF_ENOMEM;
  if ((s = ensure_copy_streams(f)) != BF_OK) return s;
  int sms = 0;
  if ((s = sm_count(f->device, &sms)) != BF_OK) return s;
  if ((s = fork_copies(f, stream)) != BF_OK) return s;
  cudaError_t e;
  uint64_t i = 0;
  int last = 0;
  for (uint64_t lo = 0; lo < n; lo += pass, ++i) {
    const int w = static_cast<int>(i & 1);
    const uint64_t cnt = std::min(pass, n - lo);
    char* base = static_cast<char*>(f->hstage) + w * slot;
    uint64_t* d_keys = reinterpret_cast<uint64_t*>(base);
    uint8_t* d_res = results_in_place ? h_out + lo : reinterpret_cast<uint8_t*>(base + kbytes);
    if (i >= 2 && (e = cudaStreamWaitEvent(f->h2d, f->ev_consumed[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if ((s = stage_keys(f, h_keys + lo, d_keys, cnt, sms, sm_copy)) != BF_OK) return s;
    if ((e = cudaEventRecord(f->ev_copied[w], f->h2d)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(stream, f->ev_copied[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if (!results_in_place && i >= 2 && (e = cudaStreamWaitEvent(stream, f->ev_drained[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if ((s = launch_lookup_pass(f, L, pl, d_keys, cnt, d_res, static_cast<char*>(f->look_ws), stream, stream,
                                f->ev_consumed[w])) != BF_OK)
      return s;
    if (results_in_place) continue;
    if ((e = cudaEventRecord(f->ev_computed[w], stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(f->d2h, f->ev_computed[w], 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
    if ((e = cudaMemcpyAsync(h_out + lo, d_res, cnt, cudaMemcpyDeviceToHost, f->d2h)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync D2H");
    if ((e = cudaEventRecord(f->ev_drained[w], f->d2h)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    last = w;
  }
  // the copy-out stream is FIFO: its last event covers every result copy
  if (!results_in_place && (e = cudaStreamWaitEvent(stream, f->ev_drained[last], 0)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamWaitEvent");
  return BF_OK;
}

// Chunked host->device pipeline of the direct kernels: chunk c runs
// entirely on stream c % depth (copy in, kernel, copy out), so its staging
// slot is reused in order; the depth-many streams overlap one chunk's copies
// with another's kernel.  The chunks never take the slice-partitioned path,
// whose workspace is one per filter.
bf_status host_chunked_direct(bf_filter* f, int op, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                              cudaStream_t stream) {
  bf_status s = ensure_pipeline(f);
  if (s != BF_OK) return s;
  cudaError_t e = cudaEventRecord(f->ev_start, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  for (int i = 0; i < kPipelineDepth; ++i)
    if ((e = cudaStreamWaitEvent(f->pipe[i], f->ev_start, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  const uint64_t per = slot_bytes(f->chunk_keys);
  uint64_t c = 0;
  for (uint64_t lo = 0; lo < n; lo += f->chunk_keys, ++c) {
    const uint64_t cnt = std::min(f->chunk_keys, n - lo);
    const int slot = static_cast<int>(c % kPipelineDepth);
    cudaStream_t st = f->pipe[slot];
    char* slot_base = static_cast<char*>(f->staging) + slot * per;
    uint64_t* d_keys = reinterpret_cast<uint64_t*>(slot_base);
    uint8_t* d_out = reinterpret_cast<uint8_t*>(slot_base + keys_region(f->chunk_keys));
    if ((e = cudaMemcpyAsync(d_keys, h_keys + lo, cnt * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync H2D");
    if ((s = launch_sbf(f, op, d_keys, cnt, op == BF_OP_ADD ? nullptr : d_out, st)) != BF_OK) return s;
    if (op == BF_OP_CONTAINS &&
        (e = cudaMemcpyAsync(h_out + lo, d_out, cnt, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync D2H");
  }
  for (int i = 0; i < kPipelineDepth; ++i) {
    if ((e = cudaEventRecord(f->ev_done[i], f->pipe[i])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(stream, f->ev_done[i], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  return BF_OK;
}

// Host-buffer entry.  Slice-partitioned work runs in passes staged through
// device memory (the staging kernel reads buffers the kernels can address,
// the copy engine the others), unless BF_HOST_DIRECT asks for in-place
// reads; otherwise Grace-coupled GPUs read host memory coherently over
// NVLink-C2C and the direct kernels stream the keys (and write the results)
// in place; else the chunked pipeline of the direct kernels.
bf_status host_pipeline(bf_filter* f, int op, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                        cudaStream_t stream) {
  const bool add = op == BF_OP_ADD;
  // kernels load keys as aligned 8-byte words; the copy engine takes any address
  const bool aligned = reinterpret_cast<uintptr_t>(h_keys) % 8 == 0;
  const bool in_place = aligned && device_can_access(f, h_keys) && (add || device_can_access(f, h_out));
  const bool part = add ? use_partitioned(f, n) : use_partitioned_lookup(f, n);
  if (part && (f->host_access != BF_HOST_DIRECT || !in_place)) {
    const bf_status s = add ? launch_partitioned_staged(f, h_keys, n, stream, in_place)
                            : launch_contains_partitioned_staged(f, h_keys, n, h_out, stream, in_place,
                                                                 in_place && !is_page_locked(h_out));
    if (s != BF_ENOMEM) return s;  // else nothing was queued: a path with less memory
  }
  if (in_place) {
    if (add) return part ? launch_partitioned_host(f, h_keys, n, stream) : run_add(f, h_keys, n, stream);
    return part ? launch_contains_partitioned_host(f, h_keys, n, h_out, stream)
                : run_contains(f, h_keys, n, h_out, stream);
  }
  return host_chunked_direct(f, op, h_keys, n, h_out, stream);
}

}  // namespace

extern "C" {

bf_status bf_params_check(const bf_params* params) {
  bf_status s = check_params(params);
  if (s != BF_OK) return s;
  bf_layout l{};
  for (int op = 0; op < 2; ++op) {
    s = resolve_layout(*params, op, nullptr, &l, nullptr);
    if (s != BF_OK) return s;
  }
  return BF_OK;
}

bf_status bf_layout_check(const bf_params* params, int op, const bf_layout* layout) {
  bf_status s = check_params(params);
  if (s != BF_OK) return s;
  bf_layout l{};
  return resolve_layout(*params, op, layout, &l, nullptr);
}

bf_status bf_create(const bf_params* params, void* d_words, bf_filter** out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  bf_status s = bf_params_check(params);
  if (s != BF_OK) return s;
  bf_filter* f = new (std::nothrow) bf_filter();
  if (!f) return fail(BF_ENOMEM, "host allocation failed");
  f->p = *params;
  f->nbytes = params->num_blocks * (params->block_bits / 8);
  cudaError_t e = cudaGetDevice(&f->device);
  if (e != cudaSuccess) {
    delete f;
    return cuda_fail(e, "cudaGetDevice");
  }
  for (int op = 0; op < 2; ++op) resolve_layout(f->p, op, nullptr, &f->layout[op], &f->entry[op]);
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, f->device);
  f->l2_bytes = static_cast<uint64_t>(l2);
  if (d_words) {
    const uint64_t align = std::max<uint64_t>(32, params->block_bits / 8);
    if (reinterpret_cast<uintptr_t>(d_words) % align != 0) {
      delete f;
      return fail(BF_EINVAL, "adopted buffer must be aligned to max(32, block_bits/8) bytes");
    }
    f->words = d_words;
    f->owned = false;
  } else {
    e = cudaMalloc(&f->words, f->nbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete f;
      return fail(BF_ENOMEM, "cudaMalloc of the bit array failed");
    }
    f->owned = true;
    e = cudaMemset(f->words, 0, f->nbytes);
    if (e != cudaSuccess) {
      cudaFree(f->words);
      delete f;
      return cuda_fail(e, "cudaMemset");
    }
  }
  *out = f;
  return BF_OK;
}

bf_status bf_destroy(bf_filter* f) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  DeviceGuard g(f->device);
  release_pipeline(f);
  if (f->part_ws) cudaFree(f->part_ws);
  if (f->look_ws) cudaFree(f->look_ws);
  if (f->status) cudaFree(f->status);
  for (cudaEvent_t e : f->ev_pool) cudaEventDestroy(e);
  if (f->owned && f->words) cudaFree(f->words);
  delete f;
  return BF_OK;
}

bf_status bf_clear(bf_filter* f, bf_stream_t stream) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  DeviceGuard g(f->device);
  cudaError_t e = cudaMemsetAsync(f->words, 0, f->nbytes, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaMemsetAsync");
}

bf_status bf_add(bf_filter* f, const uint64_t* d_keys, uint64_t n, bf_stream_t stream) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  if (n == 0) return BF_OK;
  if (!d_keys) return fail(BF_EINVAL, "keys is NULL");
  if (reinterpret_cast<uintptr_t>(d_keys) % 8) return fail(BF_EINVAL, "keys must be 8-byte aligned");
  DeviceGuard g(f->device);
  begin_call(f);
  return run_add(f, d_keys, n, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_contains(const bf_filter* f, const uint64_t* d_keys, uint64_t n, uint8_t* d_out,
                      bf_stream_t stream) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  if (n == 0) return BF_OK;
  if (!d_keys || !d_out) return fail(BF_EINVAL, "keys or out is NULL");
  if (reinterpret_cast<uintptr_t>(d_keys) % 8) return fail(BF_EINVAL, "keys must be 8-byte aligned");
  DeviceGuard g(f->device);
  begin_call(f);
  return run_contains(f, d_keys, n, d_out, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_add_host(bf_filter* f, const uint64_t* h_keys, uint64_t n, bf_stream_t stream) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  if (n == 0) return BF_OK;
  if (!h_keys) return fail(BF_EINVAL, "keys is NULL");
  DeviceGuard g(f->device);
  begin_call(f);
  return host_pipeline(f, BF_OP_ADD, h_keys, n, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_contains_host(bf_filter* f, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                           bf_stream_t stream) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  if (n == 0) return BF_OK;
  if (!h_keys || !h_out) return fail(BF_EINVAL, "keys or out is NULL");
  DeviceGuard g(f->device);
  begin_call(f);
  return host_pipeline(f, BF_OP_CONTAINS, h_keys, n, h_out, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_set_staging(bf_filter* f, uint64_t chunk_keys, int mode) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  if (chunk_keys < 1024 || chunk_keys > (1ull << 32))
    return fail(BF_EINVAL, "chunk_keys must be in [1024, 2^32]");
  if (mode != BF_HOST_AUTO && mode != BF_HOST_STAGED && mode != BF_HOST_DIRECT)
    return fail(BF_EINVAL, "mode must be BF_HOST_AUTO, BF_HOST_STAGED or BF_HOST_DIRECT");
  DeviceGuard g(f->device);
  release_pipeline(f);
  f->chunk_keys = chunk_keys;
  f->host_access = mode;
  return BF_OK;
}

bf_status bf_words(const bf_filter* f, void** d_ptr, uint64_t* nbytes) {
  if (!f || !d_ptr || !nbytes) return fail(BF_EINVAL, "NULL argument");
  *d_ptr = f->words;
  *nbytes = f->nbytes;
  return BF_OK;
}

bf_status bf_get_params(const bf_filter* f, bf_params* out) {
  if (!f || !out) return fail(BF_EINVAL, "NULL argument");
  *out = f->p;
  return BF_OK;
}

bf_status bf_set_layout(bf_filter* f, int op, const bf_layout* layout) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  bf_layout l{};
  const KernelEntry* e = nullptr;
  bf_status s = resolve_layout(f->p, op, layout, &l, &e);
  if (s != BF_OK) return s;
  f->layout[op] = l;
  f->entry[op] = e;
  return BF_OK;
}

bf_status bf_get_layout(const bf_filter* f, int op, bf_layout* out) {
  if (!f || !out) return fail(BF_EINVAL, "NULL argument");
  if (op != BF_OP_ADD && op != BF_OP_CONTAINS) return fail(BF_EINVAL, "bad op");
  *out = f->layout[op];
  return BF_OK;
}

bf_status bf_set_l2_persist(bf_filter* f, bf_stream_t stream, float hit_ratio) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  DeviceGuard g(f->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamAttrValue attr{};
  cudaError_t e;
  if (hit_ratio <= 0.f) {
    attr.accessPolicyWindow.base_ptr = nullptr;
    attr.accessPolicyWindow.num_bytes = 0;
    attr.accessPolicyWindow.hitRatio = 0.f;
    attr.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
    attr.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    if ((e = cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &attr)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamSetAttribute");
    if ((e = cudaCtxResetPersistingL2Cache()) != cudaSuccess) return cuda_fail(e, "cudaCtxResetPersistingL2Cache");
    if ((e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0)) != cudaSuccess)
      return cuda_fail(e, "cudaDeviceSetLimit");
    f->l2_window = false;
    return BF_OK;
  }
  if (hit_ratio > 1.f) hit_ratio = 1.f;
  int max_persist = 0, max_window = 0;
  cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, f->device);
  cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, f->device);
  if (max_persist <= 0 || max_window <= 0) return fail(BF_EUNSUPPORTED, "device has no L2 persistence");
  const size_t limit = std::min<uint64_t>(f->nbytes, static_cast<uint64_t>(max_persist));
  if ((e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, limit)) != cudaSuccess)
    return cuda_fail(e, "cudaDeviceSetLimit");
  attr.accessPolicyWindow.base_ptr = f->words;
  attr.accessPolicyWindow.num_bytes = std::min<uint64_t>(f->nbytes, static_cast<uint64_t>(max_window));
  attr.accessPolicyWindow.hitRatio = hit_ratio;
  attr.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  attr.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  if ((e = cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &attr)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamSetAttribute");
  f->l2_window = true;
  return BF_OK;
}

bf_status bf_gups(int mode, void* d_table, uint64_t table_bytes, uint32_t unit_bytes, const uint64_t* d_keys,
                  uint64_t n, uint8_t* d_out, const bf_layout* layout, bf_stream_t stream) {
  if (mode != BF_GUPS_LOAD && mode != BF_GUPS_RED_OR && mode != BF_GUPS_RED_OR_SECTOR)
    return fail(BF_EINVAL, "bad mode");
  if (mode == BF_GUPS_RED_OR_SECTOR && unit_bytes < 32) return fail(BF_EINVAL, "full-sector mode needs unit_bytes >= 32");
  if (unit_bytes != 8 && unit_bytes != 32 && unit_bytes != 64 && unit_bytes != 128)
    return fail(BF_EINVAL, "unit_bytes must be 8, 32, 64 or 128");
  if (!d_table || table_bytes < unit_bytes) return fail(BF_EINVAL, "table too small");
  if (reinterpret_cast<uintptr_t>(d_table) % std::max<uint32_t>(unit_bytes, 32) != 0)
    return fail(BF_EINVAL, "table must be aligned to max(32, unit_bytes)");
  if (n == 0) return BF_OK;
  if (!d_keys || (mode == BF_GUPS_LOAD && !d_out)) return fail(BF_EINVAL, "keys or out is NULL");
  if (reinterpret_cast<uintptr_t>(d_keys) % 8) return fail(BF_EINVAL, "keys must be 8-byte aligned");
  const uint32_t kpt = (layout && layout->kpt) ? layout->kpt : 2;
  const uint32_t threads = (layout && layout->block_threads) ? layout->block_threads : 256;
  const uint32_t grid_req = layout ? layout->grid_ctas : 0;
  if (threads % 32 || threads > static_cast<uint32_t>(kMaxBlockThreadsHost)) return fail(BF_EINVAL, "block_threads");
  const GupsEntry* e = find_gups(mode, unit_bytes, kpt);
  if (!e) return fail(BF_EINVAL, "kpt must be 1, 2 or 4");
  int device = 0;
  cudaError_t err = cudaGetDevice(&device);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
  uint32_t grid = 0;
  bf_status s = resolve_grid(e->fn, device, threads, grid_req, n, kpt, &grid);
  if (s != BF_OK) return s;
  const uint64_t nunits = table_bytes / unit_bytes;
  GupsArgs a{d_table, nunits, d_keys, n, d_out, nunits < (1ull << 32) ? 0 : (nunits == (1ull << 32) ? 1 : 2)};
  void* args[] = {&a};
  err = cudaLaunchKernel(e->fn, dim3(grid), dim3(threads), args, 0, reinterpret_cast<cudaStream_t>(stream));
  return err == cudaSuccess ? BF_OK : cuda_fail(err, "launch gups kernel");
}

bf_status bf_set_partition(bf_filter* f, const bf_partition* cfg) {
  if (!f || !cfg) return fail(BF_EINVAL, "NULL argument");
  if (cfg->mode > BF_PART_AUTO) return fail(BF_EINVAL, "mode must be BF_PART_OFF, BF_PART_ON or BF_PART_AUTO");
  if (cfg->slice_log2 < 16 || cfg->slice_log2 > 34) return fail(BF_EINVAL, "slice_log2 must be in [16, 34]");
  if (cfg->chunk_keys < 4096) return fail(BF_EINVAL, "chunk_keys must be >= 4096");
  if (cfg->cap_override % kRecTile) return fail(BF_EINVAL, "cap_override must be a multiple of 128");
  if (cfg->window_log2 < 16 || cfg->window_log2 > 36) return fail(BF_EINVAL, "window_log2 must be in [16, 36]");
  if (cfg->lookup_mode > BF_PART_AUTO) return fail(BF_EINVAL, "lookup_mode must be BF_PART_OFF, BF_PART_ON or BF_PART_AUTO");
  if (cfg->lookup_chunk_keys < 4096 || cfg->lookup_chunk_keys > (1ull << 32))
    return fail(BF_EINVAL, "lookup_chunk_keys must be in [4096, 2^32]");
  if (cfg->passes > 64) return fail(BF_EINVAL, "passes must be <= 64");
  if (cfg->part_ctas > 8) return fail(BF_EINVAL, "part_ctas must be <= 8");
  f->part = *cfg;
  return BF_OK;
}

bf_status bf_get_partition(const bf_filter* f, bf_partition* out) {
  if (!f || !out) return fail(BF_EINVAL, "NULL argument");
  *out = f->part;
  return BF_OK;
}

bf_status bf_last_launches(const bf_filter* f, uint32_t* n) {
  if (!f || !n) return fail(BF_EINVAL, "NULL argument");
  *n = f->last_launches;
  return BF_OK;
}

bf_status bf_device_status(bf_filter* f, bf_stream_t stream, uint32_t* codes) {
  if (!f || !codes) return fail(BF_EINVAL, "NULL argument");
  *codes = 0;
  if (!f->status) return BF_OK;  // no slice-partitioned call yet
  DeviceGuard g(f->device);
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaSuccess && f->rec_stream) e = cudaStreamSynchronize(f->rec_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  uint32_t v = 0;
  if ((e = cudaMemcpy(&v, f->status, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy(status)");
  if (v && (e = cudaMemset(f->status, 0, sizeof v)) != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
  *codes = v;
  return BF_OK;
}

bf_status bf_set_timing(bf_filter* f, int enable) {
  if (!f) return fail(BF_EINVAL, "filter is NULL");
  f->timing = enable != 0;
  f->segs.clear();
  f->ev_used = 0;
  return BF_OK;
}

bf_status bf_get_timing(bf_filter* f, bf_timing* out) {
  if (!f || !out) return fail(BF_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof *out);
  DeviceGuard g(f->device);
  for (const auto& sg : f->segs) {
    cudaError_t e = cudaEventSynchronize(sg.b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, sg.a, sg.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    out->ms[sg.phase] += ms;
    out->launches[sg.phase] += sg.launches;
  }
  f->segs.clear();
  f->ev_used = 0;
  return BF_OK;
}

const char* bf_status_str(bf_status s) {
  switch (s) {
    case BF_OK: return "BF_OK";
    case BF_EINVAL: return "BF_EINVAL";
    case BF_ENOMEM: return "BF_ENOMEM";
    case BF_ECUDA: return "BF_ECUDA";
    case BF_EUNSUPPORTED: return "BF_EUNSUPPORTED";
    case BF_ETIMEDOUT: return "BF_ETIMEDOUT";
  }
  return "unknown status";
}

const char* bf_last_error(void) { return g_last_error.c_str(); }

const char* bf_version(void) { return "bloomgb 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Construction with library-owned static scratch (no allocation per call).
//
// Some callers cannot let a library call cudaMalloc: services that give the
// GPU's memory to their own caching allocator up front (a cudaMalloc would
// then fail, or force the pool to hand memory back), and latency-critical
// loops that must not pay for cudaMalloc / cudaFree, which synchronize the
// device.  For them, bf_add_noalloc runs the slice-partitioned construction
// with its scratch (per-slice counters and slice buffers) in one file-scope
// device array, kNoAllocScratchBytes in size, that every GPU loading this
// library holds until the process exits.  The caller passes the bit array
// and the keys; nothing is allocated by a call.
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kNoAllocScratchBytes = 16ull << 20;            // 16 MiB per device
constexpr uint64_t kNoAllocStatusBytes = 256;                      // status word of the index checks
constexpr uint64_t kNoAllocCountsBytes = 8ull * kMaxParts;         // per-slice counters
constexpr uint64_t kNoAllocHeadBytes = kNoAllocStatusBytes + kNoAllocCountsBytes;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// The kernel table is built while the library loads, so that the first
// bf_add_noalloc call does not build it.
const bool g_noalloc_registry_ready = (registry(), true);

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cudaError_t noalloc_scratch(int device, void** out) {
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = ptr;
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" bf_status bf_add_noalloc(const bf_params* params, void* d_words, const uint64_t* d_keys, uint64_t n,
                                    uint64_t* max_keys, bf_stream_t stream) {
  (void)g_noalloc_registry_ready;
  if (max_keys) *max_keys = 0;
  if (!params || !d_words) return BF_EINVAL;
  if (params->groups != 0 || params->num_blocks == 0 || params->num_blocks > (1ull << 32) ||
      (params->word_bits != 32 && params->word_bits != 64) || !is_pow2(params->block_bits) ||
      params->block_bits < params->word_bits || params->block_bits > 1024)
    return BF_EINVAL;
  const uint32_t s = params->block_bits / params->word_bits;
  if (params->k < s || params->k % s != 0 || params->k > 64) return BF_EINVAL;
  if (params->salts > 1 ||
      (params->salts == 1 && !(params->block_bits == 256 && params->word_bits == 32 && params->k == 8)))
    return BF_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_words) % std::max<uint32_t>(32, params->block_bits / 8) != 0) return BF_EINVAL;
  const KernelEntry* pe = nullptr;
  const KernelEntry* re = nullptr;
  for (const auto& e : registry().sbf) {
    if (e.B != static_cast<int>(params->block_bits) || e.S != static_cast<int>(params->word_bits) ||
        e.K != static_cast<int>(params->k) || e.z != 0 || e.salts != static_cast<int>(params->salts))
      continue;
    if (e.op == 3) pe = &e;
    if (e.op == 2 && e.theta == static_cast<int>(s) && e.phi == 1 && e.kpt == 1) re = &e;
  }
  if (!pe || !re) return BF_EUNSUPPORTED;

  // slice plan of the default partitioned construction (16 MiB slices, one
  // record-insert launch per 64 MiB window)
  bf_filter plan{};
  plan.p = *params;
  plan.nbytes = params->num_blocks * (params->block_bits / 8);
  const PartPlan pl = part_plan(&plan);
  // the largest n whose slice buffers fit next to the counters
  uint64_t lo = 0, hi = kNoAllocScratchBytes / 8;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo + 1) / 2;
    if (kNoAllocHeadBytes + static_cast<uint64_t>(pl.nparts) * part_cap(&plan, pl, mid) * 8 <= kNoAllocScratchBytes)
      lo = mid;
    else
      hi = mid - 1;
  }
  if (max_keys) *max_keys = lo;
  if (n > lo) return BF_EINVAL;  // too many keys for the static scratch: split the call
  if (n == 0) return BF_OK;
  if (!d_keys || reinterpret_cast<uintptr_t>(d_keys) % 8) return BF_EINVAL;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kNoAllocMaxDevices) return BF_ECUDA;
  void* scratch = nullptr;
  if (noalloc_scratch(device, &scratch) != cudaSuccess) return BF_ECUDA;
  uint32_t* status = static_cast<uint32_t*>(scratch);
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + kNoAllocStatusBytes);
  uint64_t* records = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + kNoAllocHeadBytes);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // the array keeps the previous call's contents: the counters must start at zero
  if (cudaMemsetAsync(counts, 0, 8ull * pl.nparts, st) != cudaSuccess) return BF_ECUDA;
  const uint64_t cap = part_cap(&plan, pl, n);
  const size_t smem = partition_smem_bytes(static_cast<int>(pl.nparts));
  if (cudaFuncSetAttribute(pe->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return BF_ECUDA;
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return BF_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pe->fn, kPartThreads, smem) != cudaSuccess)
    return BF_ECUDA;
  const uint64_t tiles = (n + part_tile(false) - 1) / part_tile(false);
  PartArgs pa{d_keys, n, params->seed + 0x27D4EB2F165667C5ull + 8ull, params->num_blocks,
              params->num_blocks < (1ull << 32) ? 0 : 1, pl.shift, pl.nparts, cap, counts, records, d_words,
              nullptr, nullptr, status};
  void* pargs[] = {&pa};
  const uint32_t pgrid = static_cast<uint32_t>(std::min<uint64_t>(tiles, static_cast<uint64_t>(sms) * std::max(per_sm, 1)));
  if (cudaLaunchKernel(pe->fn, dim3(pgrid), dim3(kPartThreads), pargs, smem, st) != cudaSuccess) return BF_ECUDA;

  constexpr uint32_t kThreads = 256;
  int rper_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper_sm, re->fn, kThreads, 0) != cudaSuccess) return BF_ECUDA;
  const uint32_t slice_bytes_log2 = pl.shift + static_cast<uint32_t>(__builtin_ctz(params->block_bits / 8));
  const uint32_t per_launch = 26 > slice_bytes_log2 ? 1u << (26 - slice_bytes_log2) : 1u;
  for (uint32_t plo = 0; plo < pl.nparts; plo += per_launch) {
    const uint32_t phi = std::min(pl.nparts, plo + per_launch);
    RecArgs ra{d_words, records, counts, plo, phi, cap, 0u, params->num_blocks, status};
    const uint64_t rtiles = (static_cast<uint64_t>(phi - plo) * cap + 31) / 32;
    const uint64_t rctas = (rtiles + kThreads / 32 - 1) / (kThreads / 32);
    const uint32_t rgrid =
        static_cast<uint32_t>(std::min<uint64_t>(rctas, static_cast<uint64_t>(sms) * std::max(rper_sm, 1)));
    void* rargs[] = {&ra};
    if (cudaLaunchKernel(re->fn, dim3(rgrid), dim3(kThreads), rargs, 0, st) != cudaSuccess) return BF_ECUDA;
  }
  return BF_OK;
}

extern "C" bf_status bf_noalloc_status(uint32_t* codes) {
  if (!codes) return BF_EINVAL;
  *codes = 0;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kNoAllocMaxDevices) return BF_ECUDA;
  void* scratch = nullptr;
  if (noalloc_scratch(device, &scratch) != cudaSuccess) return BF_ECUDA;
  uint32_t v = 0;
  if (cudaMemcpy(&v, scratch, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return BF_ECUDA;
  if (v && cudaMemset(scratch, 0, sizeof v) != cudaSuccess) return BF_ECUDA;
  *codes = v;
  return BF_OK;
}

// ---------------------------------------------------------------------------
// Batched filters: many filters of one geometry in one launch per operation
// ---------------------------------------------------------------------------
struct bf_batch {
  bf_params p{};
  uint32_t nfilters = 0;
  uint64_t total_chunks = 0;
  uint64_t total_keys = 0;  // keys the batch's key array must hold
  BatchFilter* d_filters = nullptr;
  uint64_t* d_chunk_begin = nullptr;
  int device = 0;
  bf_layout layout[2]{};
  const KernelEntry* entry[2]{};
  uint32_t grid[2]{};
};

namespace {

// Resolve a batched operation's kernel and its grid (done when the layout is
// set, so that the add / contains calls only launch: capturable in a graph).
bf_status batch_resolve(bf_batch* b, int op, const bf_layout* in) {
  bf_layout l{};
  bf_status s = resolve_layout(b->p, op, in, &l, nullptr);
  if (s != BF_OK) return s;
  if (32u * l.kpt > kBatchChunk) return fail(BF_EINVAL, "kpt too large for the batch chunk");
  const KernelEntry* e = find_op(op == BF_OP_ADD ? 7 : 8, b->p, l.cg, l.phi, l.kpt);
  if (!e) return fail(BF_EUNSUPPORTED, "no batched kernel for this geometry and layout");
  uint32_t grid = 0;
  if (b->total_chunks) {
    s = resolve_grid(e->fn, b->device, l.block_threads, l.grid_ctas, b->total_chunks * 32, 1, &grid);
    if (s != BF_OK) return s;
  }
  b->layout[op] = l;
  b->entry[op] = e;
  b->grid[op] = grid;
  return BF_OK;
}

bf_status batch_launch(const bf_batch* b, int op, const uint64_t* keys, uint8_t* out, cudaStream_t stream) {
  if (b->total_chunks == 0) return BF_OK;
  const uint64_t ahead = (b->layout[op].flags & BF_HINT_PREFETCH_L2)
                            ? static_cast<uint64_t>(b->grid[op]) * (b->layout[op].block_threads / 32)
                            : 0;
  BatchArgs a{b->d_filters, b->d_chunk_begin, b->nfilters, b->total_chunks, keys, out,
              b->p.seed + 0x27D4EB2F165667C5ull + 8ull, b->layout[op].flags, ahead};
  void* args[] = {&a};
  cudaError_t e = cudaLaunchKernel(b->entry[op]->fn, dim3(b->grid[op]), dim3(b->layout[op].block_threads), args, 0,
                                   stream);
  return e == cudaSuccess ? BF_OK : cuda_fail(e, "launch batched kernel");
}

}  // namespace

extern "C" {

bf_status bf_batch_create(const bf_params* params, const bf_batch_filter* filters, uint32_t nfilters,
                          bf_batch** out) {
  if (!out) return fail(BF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params || (!filters && nfilters)) return fail(BF_EINVAL, "NULL argument");
  bf_params p = *params;
  p.num_blocks = 1;  // per filter
  bf_status s = bf_params_check(&p);
  if (s != BF_OK) return s;
  if (csbf_groups(p)) return fail(BF_EUNSUPPORTED, "batches hold sectorized filters only");
  const uint64_t align = std::max<uint64_t>(32, p.block_bits / 8);
  std::vector<BatchFilter> hf(nfilters);
  std::vector<uint64_t> begin(static_cast<size_t>(nfilters) + 1, 0);
  uint64_t total_keys = 0;
  for (uint32_t i = 0; i < nfilters; ++i) {
    const bf_batch_filter& f = filters[i];
    if (!f.d_words || reinterpret_cast<uintptr_t>(f.d_words) % align)
      return fail(BF_EINVAL, "every filter's bit array must be non-NULL and aligned to max(32, block_bits/8)");
    if (f.num_blocks == 0 || f.num_blocks > (~0ull) / 128) return fail(BF_EINVAL, "bad num_blocks in a filter");
    if (f.key_offset > (~0ull) - f.key_count) return fail(BF_EINVAL, "key range overflows");
    hf[i] = BatchFilter{f.d_words, f.num_blocks, f.key_offset, f.key_count};
    begin[i + 1] = begin[i] + (f.key_count + kBatchChunk - 1) / kBatchChunk;
    total_keys = std::max(total_keys, f.key_offset + f.key_count);
  }
  bf_batch* b = new (std::nothrow) bf_batch();
  if (!b) return fail(BF_ENOMEM, "host allocation failed");
  b->p = p;
  b->nfilters = nfilters;
  b->total_chunks = begin[nfilters];
  b->total_keys = total_keys;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess && nfilters) e = cudaMalloc(&b->d_filters, sizeof(BatchFilter) * nfilters);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_chunk_begin, sizeof(uint64_t) * (nfilters + 1));
  if (e == cudaSuccess && nfilters)
    e = cudaMemcpy(b->d_filters, hf.data(), sizeof(BatchFilter) * nfilters, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_chunk_begin, begin.data(), sizeof(uint64_t) * (nfilters + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    bf_batch_destroy(b);
    return fail(BF_ENOMEM, "device allocation for the batch failed");
  }
  for (int op = 0; op < 2; ++op) {
    if ((s = batch_resolve(b, op, nullptr)) != BF_OK) {
      bf_batch_destroy(b);
      return s;
    }
  }
  *out = b;
  return BF_OK;
}

bf_status bf_batch_destroy(bf_batch* b) {
  if (!b) return fail(BF_EINVAL, "batch is NULL");
  DeviceGuard g(b->device);
  if (b->d_filters) cudaFree(b->d_filters);
  if (b->d_chunk_begin) cudaFree(b->d_chunk_begin);
  delete b;
  return BF_OK;
}

bf_status bf_batch_set_layout(bf_batch* b, int op, const bf_layout* layout) {
  if (!b) return fail(BF_EINVAL, "batch is NULL");
  DeviceGuard g(b->device);
  return batch_resolve(b, op, layout);
}

bf_status bf_batch_get_layout(const bf_batch* b, int op, bf_layout* out) {
  if (!b || !out) return fail(BF_EINVAL, "NULL argument");
  if (op != BF_OP_ADD && op != BF_OP_CONTAINS) return fail(BF_EINVAL, "bad op");
  *out = b->layout[op];
  return BF_OK;
}

bf_status bf_batch_add(bf_batch* b, const uint64_t* d_keys, bf_stream_t stream) {
  if (!b) return fail(BF_EINVAL, "batch is NULL");
  if (b->total_chunks && (!d_keys || reinterpret_cast<uintptr_t>(d_keys) % 8))
    return fail(BF_EINVAL, "keys must be non-NULL and 8-byte aligned");
  DeviceGuard g(b->device);
  return batch_launch(b, BF_OP_ADD, d_keys, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_batch_contains(const bf_batch* b, const uint64_t* d_keys, uint8_t* d_out, bf_stream_t stream) {
  if (!b) return fail(BF_EINVAL, "batch is NULL");
  if (b->total_chunks && (!d_keys || !d_out || reinterpret_cast<uintptr_t>(d_keys) % 8))
    return fail(BF_EINVAL, "keys (8-byte aligned) and out must be non-NULL");
  DeviceGuard g(b->device);
  return batch_launch(b, BF_OP_CONTAINS, d_keys, d_out, reinterpret_cast<cudaStream_t>(stream));
}

bf_status bf_batch_info(const bf_batch* b, uint32_t* nfilters, uint64_t* total_keys) {
  if (!b) return fail(BF_EINVAL, "batch is NULL");
  if (nfilters) *nfilters = b->nfilters;
  if (total_keys) *total_keys = b->total_keys;
  return BF_OK;
}

}  // extern "C"
