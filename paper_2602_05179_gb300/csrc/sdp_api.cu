// sdp_api.cu -- the C ABI of libsdp (include/sdp.h): argument checks,
// workspace carving, kernel dispatch and the per-device status word.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "sdp_internal.cuh"

namespace sdp {

// Per-device status word: kernels OR SDP_FLAG_* bits into it.
__device__ uint32_t g_status_word;

namespace {

thread_local char g_err[512] = "";
// Optional CUDA events recorded around the dominant kernel of the calling
// thread's next operator call (sdp_set_profile_events).
thread_local cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

void prof_begin(cudaStream_t st) {
  if (g_prof_start) cudaEventRecord(g_prof_start, st);
}
void prof_end(cudaStream_t st) {
  if (g_prof_stop) cudaEventRecord(g_prof_stop, st);
  g_prof_start = g_prof_stop = nullptr;
}
// Launch shape of the dominant kernel of the calling thread's last operator
// call (sdp_last_launch).
thread_local int32_t g_last_warps = 0, g_last_ctas = 0;
void note_launch(int warps, int ctas) {
  g_last_warps = warps;
  g_last_ctas = ctas;
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SDP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------ fault injection
// One-shot host-side faults for failure-detection tests (sdp_set_fault_inject,
// or SDP_FAULT_INJECT in the environment, read at the first check).  Nothing
// here touches a device: a fault is an error code returned before the call
// launches anything, or (stall) a streaming launch whose producers never
// publish a tile, so that the DP warps' bounded waits run out.
std::mutex g_fault_mu;
bool g_fault_env_read = false;
int g_fault_alloc = 0;     // plan / search allocations left to fail
int g_fault_launch = 0;    // operator calls left to fail with SDP_ERR_CUDA
int g_fault_oom = 0;       // operator calls left to fail with SDP_ERR_OOM
uint64_t g_fault_stall_ns = 0;  // next streaming launch: producers stall, waits give up after this

int parse_faults(const char* spec) {
  // comma-separated: alloc[:N] | launch[:N] | oom[:N] | stall:NS | none
  const char* p = spec;
  while (p && *p) {
    const char* e = strchr(p, ',');
    const size_t len = e ? (size_t)(e - p) : strlen(p);
    char tok[64];
    if (len >= sizeof(tok)) return -1;
    memcpy(tok, p, len);
    tok[len] = 0;
    char* colon = strchr(tok, ':');
    long long v = 1;
    if (colon) {
      *colon = 0;
      char* end = nullptr;
      v = strtoll(colon + 1, &end, 10);
      if (!end || *end || v < 0) return -1;
    }
    if (!strcmp(tok, "alloc")) g_fault_alloc = (int)v;
    else if (!strcmp(tok, "launch")) g_fault_launch = (int)v;
    else if (!strcmp(tok, "oom")) g_fault_oom = (int)v;
    else if (!strcmp(tok, "stall") && colon) g_fault_stall_ns = (uint64_t)v;
    else if (!strcmp(tok, "none")) g_fault_alloc = g_fault_launch = g_fault_oom = 0, g_fault_stall_ns = 0;
    else return -1;
    p = e ? e + 1 : nullptr;
  }
  return 0;
}

void fault_env_locked() {
  if (g_fault_env_read) return;
  g_fault_env_read = true;
  if (const char* e = getenv("SDP_FAULT_INJECT")) parse_faults(e);
}

bool take(int& counter) {
  std::lock_guard<std::mutex> g(g_fault_mu);
  fault_env_locked();
  if (counter <= 0) return false;
  --counter;
  return true;
}

// An operator call about to launch: an injected failure, if one is pending.
int fault_call() {
  if (take(g_fault_oom)) return fail(SDP_ERR_OOM, "injected out-of-memory (SDP_FAULT_INJECT)");
  if (take(g_fault_launch)) return fail(SDP_ERR_CUDA, "injected launch failure (SDP_FAULT_INJECT)");
  return SDP_OK;
}

constexpr int kMaxDev = 64;
std::mutex g_mu;
uint32_t* g_status_ptr[kMaxDev] = {};
int g_sms[kMaxDev] = {};

int current_device(int* dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (*dev < 0 || *dev >= kMaxDev) return fail(SDP_ERR_UNSUPPORTED, "device id %d", *dev);
  return SDP_OK;
}

int status_ptr(uint32_t** out) {
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_status_word);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
    g_status_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_status_ptr[dev];
  return SDP_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The address under which the current device reads p: device or managed
// memory as is, page-locked host memory mapped for the device through its
// device pointer; NULL for memory the device cannot read.
const void* device_readable(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer;
  return nullptr;
}

// True for page-locked host memory (the device reads it over the host link).
bool is_host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// The arguments with demands replaced by their device-readable address.
sdp_split_args with_readable_demands(const sdp_split_args* a) {
  sdp_split_args b = *a;
  if (a->demands)
    b.demands = static_cast<const int32_t*>(device_readable(a->demands));
  return b;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// workspace carving (every block 256-byte aligned)
struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off = align_up(off + count * sizeof(T), 256);
    return p;
  }
};

constexpr int64_t kPlainSlots = 262144;   // PLAIN: threads in flight (grid-stride)
constexpr int64_t kFallbackSlots = 4096;  // DEQUE fallback path

// Host demands (sdp_split_eval): chunks of this many scenarios are copied
// into two device staging buffers while the previous chunk is evaluated.
constexpr int64_t kHostChunkRows = 65536;

struct SplitWs {
  int32_t* stage[2];  // host-demand staging buffers [kHostChunkRows * n], or NULL
  int64_t stage_rows;
  TourPrep prep;
  double* mean_partial;
  uint32_t* fb_count;
  uint32_t* fb_list;
  float* kscratch;
  int32_t* pscratch;
  int64_t nslots;
  unsigned long long* hist;
  unsigned char* qt;   // STREAM: narrowed demands in tour order
  uint32_t* tflags;    // STREAM: per-tile rows with a demand above Q
  unsigned long long* counter;  // PIPE: group queue (zeroed before each launch)
  uint32_t* dscratch;  // fused adjoint on TMEM: i - pred(i) per [word][lane]
  size_t bytes;
};

// AUTO: DEQUE while a demand row fits the tensor-memory staging (n bytes of
// uint8 or 2n of uint16 within 512 bytes); longer rows go to STREAM, which
// keeps 16 DP warps per SM whatever n is (measured at n = 600 / 1000:
// 0.47 / 0.77 ms against 0.78 / 2.27 ms for DEQUE's shared-memory staging);
// PLAIN where neither applies.
// soft capacity runs on the TMEM-staged deque kernel only
bool soft_deque_ok(const sdp_split_args* a) {
  return deque_supported(a->n, a->Q) && a->warps_per_cta == 0 &&
         (int64_t)a->n * (a->Q <= 254 ? 1 : 2) <= 512;
}

int resolve_algo(const sdp_split_args* a);

// The fused adjoint runs on the TMEM-staged deque kernel when the forward
// would take DEQUE in its default shape and a row fits the tensor memory.
int adjoint_tmem_warps(const sdp_split_args* a) {
  const int algo = resolve_algo(a);
  if (algo != SDP_ALGO_DEQUE && algo != SDP_ALGO_STREAM && algo != SDP_ALGO_PIPE) return 0;
  if (a->warps_per_cta != 0 || (a->ring != 0 && a->ring != 16)) return 0;
  return split_tmem_adj_warps(a->n, a->Q, a->S, num_sms());
}

// AUTO: PIPE while it supports the shape (n <= 1024, Q <= 32767, demand rows
// that bulk copies can read: 16-byte aligned device demands, or host demands
// staged into aligned buffers), hard capacity and the default launch shape;
// else the choice that sdp_split_eval_noalloc keeps (auto_algo_no_pipe).
int auto_algo_no_pipe(const sdp_split_args* a) {
  if (a->capacity_mode == SDP_CAPACITY_SOFT)
    return soft_deque_ok(a) ? SDP_ALGO_DEQUE : SDP_ALGO_PLAIN;
  if (!deque_supported(a->n, a->Q)) return SDP_ALGO_PLAIN;
  const int64_t row_bytes = (int64_t)a->n * (a->Q <= 254 ? 1 : 2);
  if (row_bytes > 512 && a->warps_per_cta == 0 && stream_supported(a->n, a->Q) &&
      (reinterpret_cast<uintptr_t>(a->demands) & 15) == 0)
    return SDP_ALGO_STREAM;
  return SDP_ALGO_DEQUE;
}

bool pipe_ok(const sdp_split_args* a) {
  if (!pipe_supported(a->n, a->Q)) return false;
  if (a->n > 0 && a->S > 0 && !is_host_ptr(a->demands) &&
      (reinterpret_cast<uintptr_t>(a->demands) & 15) != 0)
    return false;
  return true;
}

int resolve_algo(const sdp_split_args* a) {
  int algo = a->algo;
  if (algo != SDP_ALGO_AUTO) return algo;
  if (a->warps_per_cta == 0 && (a->ring == 0 || a->ring == 16) && pipe_ok(a)) return SDP_ALGO_PIPE;
  return auto_algo_no_pipe(a);
}

SplitWs carve_split(const sdp_split_args* a, void* base, bool backward) {
  SplitWs w{};
  Carver c{static_cast<unsigned char*>(base)};
  const int n = a->n;
  const int algo = resolve_algo(a);
  w.prep.rec = c.take<StepRec>((size_t)n);
  w.prep.cols = c.take<uint16_t>((size_t)n);
  w.prep.Dn = c.take<double>(1);
  w.mean_partial = c.take<double>(kMeanBlocks);
  w.fb_count = c.take<uint32_t>(1);
  if (algo == SDP_ALGO_DEQUE || algo == SDP_ALGO_STREAM || algo == SDP_ALGO_PIPE) {
    w.fb_list = c.take<uint32_t>((size_t)a->S);
    w.nslots = a->S < kFallbackSlots ? a->S : kFallbackSlots;
  } else {
    w.fb_list = nullptr;
    w.nslots = a->S < kPlainSlots ? a->S : kPlainSlots;
  }
  if (w.nslots < 1) w.nslots = 1;
  w.kscratch = c.take<float>((size_t)(n + 1) * w.nslots);
  w.pscratch = backward ? c.take<int32_t>((size_t)n * w.nslots) : nullptr;
  w.hist = backward ? c.take<unsigned long long>(2 * (size_t)n + 1) : nullptr;
  w.dscratch = (backward && adjoint_tmem_warps(a) > 0)
                   ? c.take<uint32_t>(split_tmem_adj_scratch_bytes(n, a->Q, num_sms()) / 4)
                   : nullptr;
  w.qt = nullptr;
  w.tflags = nullptr;
  w.counter = nullptr;
  if (algo == SDP_ALGO_PIPE && !backward && n > 0) {
    const int64_t rows = (n > 0 && is_host_ptr(a->demands))
                             ? (a->S < kHostChunkRows ? a->S : kHostChunkRows)
                             : a->S;
    w.qt = c.take<unsigned char>(pipe_ring_bytes(n, a->Q, rows, 1, false));
    w.counter = c.take<unsigned long long>(1);
  }
  if (algo == SDP_ALGO_STREAM && !backward && n > 0) {
    const int64_t rows = (n > 0 && is_host_ptr(a->demands))
                             ? (a->S < kHostChunkRows ? a->S : kHostChunkRows)
                             : a->S;
    w.qt = c.take<unsigned char>(stream_qt_bytes(n, a->Q, rows));
    w.tflags = c.take<uint32_t>((size_t)((rows + 31) / 32));
  }
  w.stage[0] = w.stage[1] = nullptr;
  w.stage_rows = 0;
  if (!backward && n > 0 && a->S > 0 && is_host_ptr(a->demands)) {
    w.stage_rows = a->S < kHostChunkRows ? a->S : kHostChunkRows;
    w.stage[0] = c.take<int32_t>((size_t)w.stage_rows * n);
    w.stage[1] = c.take<int32_t>((size_t)w.stage_rows * n);
  }
  w.bytes = c.off;
  return w;
}

int run_split_core(const sdp_split_args* a, const SplitWs& w, uint32_t* status,
                   unsigned long long* hist, cudaStream_t st);

// Copy stream and events of the host-demand pipeline, made once per device on
// first use and kept for the life of the process.
struct HostPipe {
  cudaStream_t copy = nullptr;
  cudaEvent_t start = nullptr, ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
};
HostPipe g_pipe[kMaxDev];
std::mutex g_pipe_mu;

// Split with demands in page-locked host memory: chunk k is copied on the
// pipeline's copy stream into staging buffer k % 2 while chunk k - 1 runs on
// the caller's stream; copy k waits for the evaluation of chunk k - 2, which
// read the same buffer.  The caller's stream ends with every chunk evaluated.
int run_split_host_chunks(const sdp_split_args* a, const SplitWs& w, uint32_t* status,
                          cudaStream_t st) {
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe& hp = g_pipe[dev];
  if (!hp.copy) {
    cudaError_t e = cudaStreamCreateWithFlags(&hp.copy, cudaStreamNonBlocking);
    for (int b = 0; e == cudaSuccess && b < 2; ++b) {
      e = cudaEventCreateWithFlags(&hp.ready[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.done[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.start, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "host pipeline setup");
  }
  // the staging buffers may still be read by earlier work on the caller's stream
  cudaError_t e = cudaEventRecord(hp.start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.copy, hp.start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "host pipeline start");
  const int n = a->n;
  const size_t pbytes = a->pred_dtype == SDP_PRED_U16 ? 2 : 4;
  int k = 0;
  for (int64_t s0 = 0; s0 < a->S; s0 += w.stage_rows, ++k) {
    const int b = k & 1;
    const int64_t cnt = a->S - s0 < w.stage_rows ? a->S - s0 : w.stage_rows;
    if (k >= 2) e = cudaStreamWaitEvent(hp.copy, hp.done[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.stage[b], a->demands + s0 * n, sizeof(int32_t) * (size_t)cnt * n,
                          cudaMemcpyHostToDevice, hp.copy);
    if (e == cudaSuccess) e = cudaEventRecord(hp.ready[b], hp.copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, hp.ready[b], 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.fb_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "host pipeline copy");
    sdp_split_args c = *a;
    c.S = cnt;
    c.demands = w.stage[b];
    c.cost_out = a->cost_out + s0;
    if (a->pred_out)
      c.pred_out = static_cast<unsigned char*>(a->pred_out) + (size_t)s0 * n * pbytes;
    rc = run_split_core(&c, w, status, nullptr, st);
    if (rc) return rc;
    e = cudaEventRecord(hp.done[b], st);
    if (e != cudaSuccess) return cuda_fail(e, "host pipeline record");
  }
  return SDP_OK;
}

int check_split(const sdp_split_args* a, bool need_cost) {
  if (!a) return fail(SDP_ERR_INVALID_ARG, "args is NULL");
  if (a->n < 0) return fail(SDP_ERR_INVALID_ARG, "n = %d < 0", a->n);
  if (a->Q <= 0) return fail(SDP_ERR_INVALID_ARG, "Q = %d <= 0", a->Q);
  if (a->S < 0) return fail(SDP_ERR_INVALID_ARG, "S = %lld < 0", (long long)a->S);
  if (a->S > (int64_t)0xFFFFFFFFll) return fail(SDP_ERR_UNSUPPORTED, "S above 2^32-1");
  if (a->algo < SDP_ALGO_AUTO || a->algo > SDP_ALGO_PIPE)
    return fail(SDP_ERR_INVALID_ARG, "unknown algo %d", a->algo);
  if (a->algo == SDP_ALGO_PIPE && !pipe_supported(a->n, a->Q))
    return fail(SDP_ERR_UNSUPPORTED, "PIPE needs 1 <= n <= %d and Q <= 32767", kPipeMaxN);
  if (a->algo == SDP_ALGO_PIPE && a->n > 0 && a->S > 0 && !is_host_ptr(a->demands) &&
      (reinterpret_cast<uintptr_t>(a->demands) & 15))
    return fail(SDP_ERR_UNSUPPORTED, "PIPE needs 16-byte aligned demands");
  if (a->algo == SDP_ALGO_DEQUE && !deque_supported(a->n, a->Q))
    return fail(SDP_ERR_UNSUPPORTED, "DEQUE needs 1 <= n <= 65534 and Q <= 32767");
  if (a->algo == SDP_ALGO_STREAM && !stream_supported(a->n, a->Q))
    return fail(SDP_ERR_UNSUPPORTED, "STREAM needs 1 <= n <= %d and Q <= 32767", kStreamMaxN);
  if (a->algo == SDP_ALGO_STREAM && (reinterpret_cast<uintptr_t>(a->demands) & 15))
    return fail(SDP_ERR_UNSUPPORTED, "STREAM needs 16-byte aligned demands");
  if (a->capacity_mode != SDP_CAPACITY_HARD && a->capacity_mode != SDP_CAPACITY_SOFT)
    return fail(SDP_ERR_INVALID_ARG, "unknown capacity_mode %d", a->capacity_mode);
  if (a->capacity_mode == SDP_CAPACITY_SOFT) {
    if (!(a->overload_penalty >= 0.f) || a->overload_penalty == INFINITY)
      return fail(SDP_ERR_INVALID_ARG, "overload_penalty must be finite and >= 0");
    if (a->algo == SDP_ALGO_STREAM)
      return fail(SDP_ERR_UNSUPPORTED, "soft capacity runs on PLAIN, DEQUE or PIPE");
    if (a->algo == SDP_ALGO_DEQUE && !soft_deque_ok(a))
      return fail(SDP_ERR_UNSUPPORTED,
                  "soft-capacity DEQUE needs rows of at most 512 bytes and warps_per_cta = 0");
  }
  if (need_cost && a->S > 0 && !is_device_ptr(a->cost_out))
    return fail(SDP_ERR_INVALID_ARG, "cost_out must be a device pointer");
  if (a->n > 0 && a->S > 0) {
    if ((a->coords == nullptr) == (a->dist == nullptr))
      return fail(SDP_ERR_INVALID_ARG, "exactly one of coords / dist must be set");
    if (!is_device_ptr(a->tour)) return fail(SDP_ERR_INVALID_ARG, "tour must be a device pointer");
    if (a->coords && !is_device_ptr(a->coords))
      return fail(SDP_ERR_INVALID_ARG, "coords must be a device pointer");
    if (a->dist && !is_device_ptr(a->dist))
      return fail(SDP_ERR_INVALID_ARG, "dist must be a device pointer");
    if (!device_readable(a->demands))
      return fail(SDP_ERR_INVALID_ARG,
                  "demands must be device memory or page-locked host memory mapped for the device");
  }
  if (a->pred_out) {
    if (a->pred_dtype != SDP_PRED_U16 && a->pred_dtype != SDP_PRED_I32)
      return fail(SDP_ERR_INVALID_ARG, "pred_dtype must be SDP_PRED_U16 or SDP_PRED_I32");
    if (a->pred_dtype == SDP_PRED_U16 && a->n >= 65535)
      return fail(SDP_ERR_UNSUPPORTED, "uint16 predecessors need n < 65535");
    if (a->S > 0 && a->n > 0 && !is_device_ptr(a->pred_out))
      return fail(SDP_ERR_INVALID_ARG, "pred_out must be a device pointer");
  }
  if (a->mean_out && !is_device_ptr(a->mean_out))
    return fail(SDP_ERR_INVALID_ARG, "mean_out must be a device pointer");
  if (a->warps_per_cta < 0 || a->warps_per_cta > 8)
    return fail(SDP_ERR_INVALID_ARG, "warps_per_cta must be 0..8");
  if (a->ring != 0 && a->ring != 8 && a->ring != 16 && a->ring != 32)
    return fail(SDP_ERR_INVALID_ARG, "ring must be 0, 8, 16 or 32");
  return SDP_OK;
}

int check_ws(void* ws, size_t have, size_t need) {
  if (need == 0) return SDP_OK;
  if (!ws || have < need)
    return fail(SDP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, have);
  if (!is_device_ptr(ws)) return fail(SDP_ERR_INVALID_ARG, "workspace must be a device pointer");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(SDP_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  return SDP_OK;
}

// Runs the chosen DP kernel over all S, then recomputes the scenarios it
// flagged (one warp each where split_rescue.cu applies: hard capacity, no
// route histogram; else the plain kernel over the flagged list), or runs the
// PLAIN kernel over all S.
int run_split_core(const sdp_split_args* a, const SplitWs& w, uint32_t* status,
                   unsigned long long* hist, cudaStream_t st) {
  int algo = resolve_algo(a);
  if ((algo == SDP_ALGO_STREAM || algo == SDP_ALGO_PIPE) && hist)
    algo = SDP_ALGO_DEQUE;  // the fused adjoint is DEQUE's
  const int sms = num_sms();
  float* cost = hist ? nullptr : a->cost_out;
  void* pred = hist ? nullptr : a->pred_out;
  if (algo == SDP_ALGO_STREAM) {
    StreamArgs sa{};
    sa.n = a->n; sa.Q = a->Q; sa.S = a->S;
    sa.rec = w.prep.rec; sa.cols = w.prep.cols; sa.Dn = w.prep.Dn;
    sa.demands = a->demands; sa.qt = w.qt; sa.stride = stream_row_stride(a->n, a->Q);
    sa.tflags = w.tflags; sa.cost = cost; sa.pred = pred; sa.pred_dtype = a->pred_dtype;
    sa.fb_list = w.fb_list; sa.fb_count = w.fb_count; sa.status = status;
    sa.ctas_per_sm = 0;
    const uint64_t stall = fault_stall_ns();
    sa.wait_ns = stall ? stall : kWaitLimitNs;
    sa.stall = stall ? 1 : 0;
    note_launch(0, 0);
    prof_begin(st);  // both kernels of the path: pre-pass + DP
    const int e = launch_split_stream(sa, st);
    prof_end(st);
    if (e) return cuda_fail((cudaError_t)e, "split_stream launch");
  }
  if (algo == SDP_ALGO_PIPE) {
    PipeArgs pa{};
    pa.batched = 0;
    pa.B = 1; pa.Q = a->Q; pa.S = a->S; pa.n1 = a->n;
    pa.cols = w.prep.cols; pa.rec = w.prep.rec; pa.Dn = w.prep.Dn;
    pa.demands = a->demands; pa.cost = cost; pa.pred = pred; pa.pred_dtype = a->pred_dtype;
    pa.qt = w.qt; pa.stride = pipe_row_stride(a->n, a->Q); pa.counter = w.counter;
    pa.fb_count = w.fb_count; pa.fb_list1 = w.fb_list; pa.status = status;
    pa.soft = a->capacity_mode == SDP_CAPACITY_SOFT ? 1 : 0; pa.beta = a->overload_penalty;
    const uint64_t stall = fault_stall_ns();
    pa.wait_ns = stall ? stall : kWaitLimitNs;
    pa.stall = stall ? 1 : 0;
    cudaError_t ce = cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), st);
    if (ce != cudaSuccess) return cuda_fail(ce, "pipe counter reset");
    note_launch(32, pipe_grid(a->S, 1, false));  // 23 DP + 1 issuing + 8 narrowing warps
    prof_begin(st);
    const int e = launch_split_pipe(pa, st);
    prof_end(st);
    if (e) return cuda_fail((cudaError_t)e, "split_pipe launch");
  }
  const int adj_warps = (hist && w.dscratch) ? adjoint_tmem_warps(a) : 0;
  if (algo == SDP_ALGO_DEQUE && adj_warps > 0) {
    SplitDequeArgs d{};
    d.n = a->n; d.Q = a->Q; d.S = a->S;
    d.rec = w.prep.rec; d.cols = w.prep.cols; d.Dn = w.prep.Dn;
    d.demands = a->demands; d.cost = nullptr; d.pred = nullptr; d.pred_dtype = a->pred_dtype;
    d.hist = hist; d.fb_list = w.fb_list; d.fb_count = w.fb_count; d.status = status;
    note_launch(adj_warps, sms);
    prof_begin(st);
    const int e = launch_split_tmem_adj(d, adj_warps, w.dscratch, sms, st);
    prof_end(st);
    if (e) return cuda_fail((cudaError_t)e, "split_tmem_adj launch");
  } else if (algo == SDP_ALGO_DEQUE) {
    const int ring = a->ring > 0 ? a->ring : 16;
    const int pbytes = pred ? (a->pred_dtype == SDP_PRED_U16 ? 2 : 4) : 0;
    // warps_per_cta == 0: default launch, TMEM staging when the rows fit;
    // an explicit warp count selects shared-memory staging with that shape.
    DequeConfig cfg = deque_config(a->n, a->Q, a->warps_per_cta, ring, hist != nullptr, pbytes,
                                   a->warps_per_cta == 0);
    if (a->warps_per_cta == 0 && !hist && a->capacity_mode != SDP_CAPACITY_SOFT) {
      const bool direct_ok = !pred || ((a->n & 3) == 0 && (reinterpret_cast<uintptr_t>(pred) & 15) == 0);
      cfg = deque_config_wide(cfg, a->n, a->Q, a->S, direct_ok, sms);
    }
    const int warps = cfg.warps;
    if (cfg.smem > 227 * 1024)
      return fail(SDP_ERR_UNSUPPORTED, "DEQUE tile needs %zu B of shared memory; lower warps_per_cta", cfg.smem);
    int occ = 0;
    int e = deque_max_ctas_per_sm(cfg, hist != nullptr, a->pred_dtype, pred != nullptr, &occ);
    if (e) return cuda_fail((cudaError_t)e, "deque occupancy");
    if (occ < 1) return fail(SDP_ERR_UNSUPPORTED, "DEQUE configuration does not fit on an SM");
    const int64_t tiles = (a->S + 31) / 32;
    const int64_t ctas_needed = (tiles + warps - 1) / warps;
    const int grid = (int)(ctas_needed < (int64_t)occ * sms ? ctas_needed : (int64_t)occ * sms);
    SplitDequeArgs d{};
    d.n = a->n; d.Q = a->Q; d.S = a->S;
    d.rec = w.prep.rec; d.cols = w.prep.cols; d.Dn = w.prep.Dn;
    d.demands = a->demands; d.cost = cost; d.pred = pred; d.pred_dtype = a->pred_dtype;
    d.hist = hist; d.fb_list = w.fb_list; d.fb_count = w.fb_count; d.status = status;
    d.soft = a->capacity_mode == SDP_CAPACITY_SOFT; d.beta = a->overload_penalty;
    note_launch(warps, grid);
    prof_begin(st);
    e = launch_split_deque(d, cfg, grid, st);
    prof_end(st);
    if (e) return cuda_fail((cudaError_t)e, "split_deque launch");
  }
  if (algo != SDP_ALGO_PLAIN && !hist && a->capacity_mode != SDP_CAPACITY_SOFT &&
      rescue_supported(a->n)) {
    // the scenarios the DP kernel flagged, one warp each
    RescueArgs r{};
    r.batched = 0; r.Q = a->Q; r.S = a->S; r.n_max = a->n; r.n1 = a->n;
    r.fb_list1 = w.fb_list; r.cost = cost; r.pred = pred; r.pred_dtype = a->pred_dtype;
    r.rec = w.prep.rec; r.Dn = w.prep.Dn; r.demands = a->demands;
    r.fb_count = w.fb_count; r.status = status;
    const int e = launch_split_rescue(r, a->S, st);
    if (e) return cuda_fail((cudaError_t)e, "split_rescue launch");
    return SDP_OK;
  }
  SplitPlainArgs p{};
  p.n = a->n; p.Q = a->Q; p.S = a->S;
  p.rec = w.prep.rec; p.Dn = w.prep.Dn; p.demands = a->demands;
  p.cost = cost; p.pred = pred; p.pred_dtype = a->pred_dtype;
  p.kscratch = w.kscratch; p.pscratch = (hist && !pred) ? w.pscratch : nullptr;
  p.nslots = w.nslots; p.hist = hist;
  p.fb_list = algo != SDP_ALGO_PLAIN ? w.fb_list : nullptr;
  p.fb_count = w.fb_count; p.status = status;
  p.soft = a->capacity_mode == SDP_CAPACITY_SOFT; p.beta = a->overload_penalty;
  const int grid = (int)((w.nslots + 255) / 256);
  if (algo == SDP_ALGO_PLAIN) {
    note_launch(8, grid);
    prof_begin(st);
  }
  launch_split_plain(p, grid, st);
  if (algo == SDP_ALGO_PLAIN) prof_end(st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "split_plain launch");
  return SDP_OK;
}

}  // namespace

int status_word(uint32_t** out) { return status_ptr(out); }

bool fault_alloc() { return take(g_fault_alloc); }

uint64_t fault_stall_ns() {
  std::lock_guard<std::mutex> g(g_fault_mu);
  fault_env_locked();
  const uint64_t v = g_fault_stall_ns;
  g_fault_stall_ns = 0;
  return v;
}

int fault_call_hook() { return fault_call(); }

int api_fail(int code, const char* msg) { return fail(code, "%s", msg); }

bool api_device_ptr(const void* p) { return is_device_ptr(p); }

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
  if (!g_sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = v > 0 ? v : 1;
  }
  return g_sms[dev];
}

}  // namespace sdp

using namespace sdp;

extern "C" {

int sdp_version(void) { return SDP_VERSION; }

const char* sdp_last_error(void) { return g_err; }

size_t sdp_split_args_size(void) { return sizeof(sdp_split_args); }

int sdp_set_profile_events(void* start, void* stop) {
  if ((start == nullptr) != (stop == nullptr))
    return fail(SDP_ERR_INVALID_ARG, "give both events or neither");
  g_prof_start = static_cast<cudaEvent_t>(start);
  g_prof_stop = static_cast<cudaEvent_t>(stop);
  return SDP_OK;
}
int sdp_set_fault_inject(const char* spec) {
  std::lock_guard<std::mutex> g(g_fault_mu);
  g_fault_env_read = true;  // an explicit setting replaces the environment's
  g_fault_alloc = g_fault_launch = g_fault_oom = 0;
  g_fault_stall_ns = 0;
  if (spec && parse_faults(spec)) {
    g_fault_alloc = g_fault_launch = g_fault_oom = 0;
    g_fault_stall_ns = 0;
    return fail(SDP_ERR_INVALID_ARG, "bad fault spec '%s'", spec);
  }
  return SDP_OK;
}

int sdp_last_launch(int32_t* warps_per_cta_out, int32_t* ctas_out) {
  if (warps_per_cta_out) *warps_per_cta_out = g_last_warps;
  if (ctas_out) *ctas_out = g_last_ctas;
  return SDP_OK;
}
size_t sdp_reinsert_args_size(void) { return sizeof(sdp_reinsert_args); }

int sdp_device_status(int clear, uint32_t* flags_out) {
  uint32_t* sp;
  int rc = status_ptr(&sp);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  uint32_t v = 0;
  e = cudaMemcpy(&v, sp, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  if (clear) {
    e = cudaMemset(sp, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
  }
  if (flags_out) *flags_out = v;
  if (v & SDP_FLAG_DEVICE_CHECK) return fail(SDP_ERR_DEVICE_CHECK, "a kernel bounds check fired");
  return (v & SDP_FLAG_INFEASIBLE) ? SDP_WARN_INFEASIBLE : SDP_OK;
}

size_t sdp_split_workspace_bytes(const sdp_split_args* a) {
  if (!a || a->n < 0 || a->S < 0) return 0;
  return carve_split(a, nullptr, false).bytes;
}

size_t sdp_split_backward_workspace_bytes(const sdp_split_args* a) {
  if (!a || a->n < 0 || a->S < 0) return 0;
  return carve_split(a, nullptr, true).bytes;
}

int sdp_split_eval(const sdp_split_args* args, void* stream) {
  int rc = check_split(args, true);
  if (rc) return rc;
  const sdp_split_args rd = with_readable_demands(args);
  const sdp_split_args* a = &rd;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SplitWs need = carve_split(a, nullptr, false);
  rc = check_ws(a->workspace, a->workspace_bytes, need.bytes);
  if (rc) return rc;
  uint32_t* status;
  rc = status_ptr(&status);
  if (rc) return rc;
  rc = fault_call();
  if (rc) return rc;
  const SplitWs w = carve_split(a, a->workspace, false);
  if (a->S > 0 && a->n == 0) {
    cudaError_t e = cudaMemsetAsync(a->cost_out, 0, sizeof(float) * a->S, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset cost");
  } else if (a->S > 0) {
    launch_tour_prep(a->tour, a->n, a->coords, a->dist, w.prep, status, w.fb_count, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tour_prep launch");
    // host demands: copied chunk by chunk (from the caller's host address)
    // behind the evaluation of the previous chunk
    rc = w.stage_rows > 0 ? run_split_host_chunks(args, w, status, st)
                          : run_split_core(a, w, status, nullptr, st);
    if (rc) return rc;
  }
  if (a->mean_out) {
    launch_mean(a->cost_out, a->S, w.mean_partial, a->mean_out, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mean launch");
  }
  return SDP_OK;
}

}  // extern "C"

// ------------------------------------------------------------ no-allocation
// Fixed device scratch for sdp_split_eval_noalloc.  Every device that loads
// this library holds these SDP_NOALLOC_SCRATCH_BYTES until the process exits.
// In host code the symbol is only a host-side handle: kernels receive the
// device address obtained below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SDP_NOALLOC_SCRATCH_BYTES];

namespace {
void* g_noalloc_ptr[kMaxDev] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
int noalloc_scratch(void** out) {
  int dev;
  int rc = current_device(&dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SDP_OK;
}
}  // namespace

extern "C" {

int sdp_split_eval_noalloc(const sdp_split_args* a, void* stream) {
  if (!a) return fail(SDP_ERR_INVALID_ARG, "args is NULL");
  if (a->n < 0 || a->S < 0) return fail(SDP_ERR_INVALID_ARG, "n and S must be >= 0");
  // AUTO keeps its choice without PIPE here: PIPE's slot ring (tens of MB)
  // would not fit the fixed scratch at the sizes this entry point serves
  sdp_split_args b = *a;
  if (b.algo == SDP_ALGO_AUTO) b.algo = auto_algo_no_pipe(a);
  const size_t need = sdp_split_workspace_bytes(&b);
  if (need > (size_t)SDP_NOALLOC_SCRATCH_BYTES)
    return fail(SDP_ERR_UNSUPPORTED,
                "this call needs %zu bytes of scratch; the no-allocation scratch holds %zu "
                "(use sdp_split_eval with a caller workspace)",
                need, (size_t)SDP_NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  b.workspace = scratch;
  b.workspace_bytes = SDP_NOALLOC_SCRATCH_BYTES;
  return sdp_split_eval(&b, stream);
}

// ------------------------------------------------------ fleet-limited Split
}  // extern "C"

namespace {
struct FleetWs {
  TourPrep prep;
  double* mean_partial;
  uint32_t* fb_count;
  uint32_t* fb_list;
  float* kscratch;
  uint16_t* pscratch;
  uint16_t* dscratch;
  int64_t nslots;
  FleetConfig cfg;
  size_t bytes;
};
constexpr int64_t kFleetPlainSlots = 65536;   // PLAIN: scenarios in flight
constexpr int64_t kFleetFallbackSlots = 1024; // recomputation of flagged scenarios

FleetWs carve_fleet(const sdp_split_args* a, int K, bool routes, void* base) {
  FleetWs w{};
  Carver c{static_cast<unsigned char*>(base)};
  const int n = a->n;
  const bool plain = a->algo == SDP_ALGO_PLAIN;
  w.prep.rec = c.take<StepRec>((size_t)n);
  w.prep.cols = c.take<uint16_t>((size_t)n);
  w.prep.Dn = c.take<double>(1);
  w.mean_partial = c.take<double>(kMeanBlocks);
  w.fb_count = c.take<uint32_t>(1);
  w.fb_list = plain ? nullptr : c.take<uint32_t>((size_t)a->S);
  const int64_t cap = plain ? kFleetPlainSlots : kFleetFallbackSlots;
  w.nslots = a->S < cap ? a->S : cap;
  if (w.nslots < 1) w.nslots = 1;
  w.kscratch = c.take<float>((size_t)w.nslots * 2 * (size_t)(n + 1));
  w.pscratch = routes ? c.take<uint16_t>((size_t)w.nslots * K * (size_t)n) : nullptr;
  w.cfg = plain || n == 0 ? FleetConfig{} : fleet_config(n, K, a->S);
  w.dscratch = (routes && !plain && n > 0) ? c.take<uint16_t>(fleet_dscratch_elems(n, K, w.cfg))
                                          : nullptr;
  w.bytes = c.off;
  return w;
}

int check_fleet(const sdp_split_args* a, int32_t K) {
  int rc = check_split(a, true);
  if (rc) return rc;
  if (K < 1 || K > kFleetMaxK) return fail(SDP_ERR_UNSUPPORTED, "max_routes = %d outside 1..%d", K, kFleetMaxK);
  if (a->n > 16384) return fail(SDP_ERR_UNSUPPORTED, "fleet-limited Split needs n <= 16384");
  if (a->Q > 32767) return fail(SDP_ERR_UNSUPPORTED, "fleet-limited Split needs Q <= 32767");
  if (a->capacity_mode != SDP_CAPACITY_HARD)
    return fail(SDP_ERR_UNSUPPORTED, "fleet-limited Split takes hard capacity");
  if (a->pred_out) return fail(SDP_ERR_INVALID_ARG, "fleet-limited Split returns routes, not pred_out");
  if (a->algo != SDP_ALGO_AUTO && a->algo != SDP_ALGO_PLAIN)
    return fail(SDP_ERR_UNSUPPORTED, "fleet-limited Split takes algo AUTO or PLAIN");
  if (a->n > 0 && a->S > 0 && !is_device_ptr(a->demands))
    return fail(SDP_ERR_INVALID_ARG, "fleet-limited Split needs device demands");
  return SDP_OK;
}
}  // namespace

extern "C" {

size_t sdp_split_fleet_workspace_bytes(const sdp_split_args* a, int32_t max_routes,
                                       int32_t want_routes) {
  if (!a || a->n < 0 || a->S < 0 || max_routes < 1 || max_routes > kFleetMaxK) return 0;
  return carve_fleet(a, max_routes, want_routes != 0, nullptr).bytes;
}

int sdp_split_fleet_eval(const sdp_split_args* a, int32_t max_routes, int32_t* nroutes_out,
                         uint8_t* route_out, void* stream) {
  int rc = check_fleet(a, max_routes);
  if (rc) return rc;
  if (nroutes_out && a->S > 0 && !is_device_ptr(nroutes_out))
    return fail(SDP_ERR_INVALID_ARG, "nroutes_out must be a device pointer");
  if (route_out && a->S > 0 && a->n > 0 && !is_device_ptr(route_out))
    return fail(SDP_ERR_INVALID_ARG, "route_out must be a device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool routes = route_out != nullptr && a->n > 0;
  const FleetWs need = carve_fleet(a, max_routes, routes, nullptr);
  rc = check_ws(a->workspace, a->workspace_bytes, need.bytes);
  if (rc) return rc;
  uint32_t* status;
  rc = status_ptr(&status);
  if (rc) return rc;
  rc = fault_call();
  if (rc) return rc;
  const FleetWs w = carve_fleet(a, max_routes, routes, a->workspace);
  if (a->S > 0 && a->n == 0) {
    cudaError_t e = cudaMemsetAsync(a->cost_out, 0, sizeof(float) * a->S, st);
    if (e == cudaSuccess && nroutes_out) e = cudaMemsetAsync(nroutes_out, 0, sizeof(int32_t) * a->S, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset fleet outputs");
  } else if (a->S > 0) {
    launch_tour_prep(a->tour, a->n, a->coords, a->dist, w.prep, status, w.fb_count, st);
    SplitFleetArgs f{};
    f.n = a->n; f.Q = a->Q; f.K = max_routes; f.S = a->S;
    f.rec = w.prep.rec; f.Dn = w.prep.Dn; f.demands = a->demands;
    f.cost = a->cost_out; f.nroutes = nroutes_out; f.route = routes ? route_out : nullptr;
    f.fb_count = w.fb_count; f.status = status;
    f.kscratch = w.kscratch; f.pscratch = w.pscratch; f.nslots = w.nslots;
    int e = 0;
    if (a->algo == SDP_ALGO_PLAIN) {
      f.fb_list = nullptr;  // every scenario
      note_launch(8, (int)((w.nslots + 255) / 256));
      prof_begin(st);
      e = launch_split_fleet_plain(f, st);
      prof_end(st);
      if (e) return cuda_fail((cudaError_t)e, "split_fleet_plain launch");
    } else {
      f.fb_list = w.fb_list;
      f.dscratch = w.dscratch;
      note_launch(w.cfg.warps, w.cfg.grid);
      prof_begin(st);
      e = launch_split_fleet(f, w.cfg, st);
      prof_end(st);
      if (e) return cuda_fail((cudaError_t)e, "split_fleet launch");
      // the flagged scenarios, if any
      e = fleet_rescue_supported(a->n) ? launch_split_fleet_rescue(f, st) : launch_split_fleet_plain(f, st);
      if (e) return cuda_fail((cudaError_t)e, "split_fleet recompute launch");
    }
  }
  if (a->mean_out) {
    launch_mean(a->cost_out, a->S, w.mean_partial, a->mean_out, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mean launch");
  }
  return SDP_OK;
}

int sdp_split_count_arcs(const sdp_split_args* args, int64_t* arcs_out, uint64_t* total_out,
                         void* stream) {
  int rc = check_split(args, false);
  if (rc) return rc;
  const sdp_split_args rd = with_readable_demands(args);
  const sdp_split_args* a = &rd;
  if (arcs_out && !is_device_ptr(arcs_out)) return fail(SDP_ERR_INVALID_ARG, "arcs_out must be a device pointer");
  if (total_out && !is_device_ptr(total_out)) return fail(SDP_ERR_INVALID_ARG, "total_out must be a device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SplitWs need = carve_split(a, nullptr, false);
  rc = check_ws(a->workspace, a->workspace_bytes, need.bytes);
  if (rc) return rc;
  uint32_t* status;
  rc = status_ptr(&status);
  if (rc) return rc;
  const SplitWs w = carve_split(a, a->workspace, false);
  if (total_out) {
    cudaError_t e = cudaMemsetAsync(total_out, 0, sizeof(uint64_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "memset total");
  }
  if (a->S == 0) return SDP_OK;
  if (a->n == 0) {
    if (arcs_out) {
      cudaError_t e = cudaMemsetAsync(arcs_out, 0, sizeof(int64_t) * a->S, st);
      if (e != cudaSuccess) return cuda_fail(e, "memset arcs");
    }
    return SDP_OK;
  }
  launch_tour_prep(a->tour, a->n, a->coords, a->dist, w.prep, status, w.fb_count, st);
  launch_count_arcs(a->n, a->Q, a->S, w.prep.rec, a->demands, arcs_out,
                    reinterpret_cast<unsigned long long*>(total_out), 4 * num_sms(), st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "count_arcs launch");
  return SDP_OK;
}

int sdp_split_backward(const sdp_split_args* args, const void* pred, const float* grad_mean,
                       float* grad_dist, int64_t* route_hist_out, void* stream) {
  int rc = check_split(args, false);
  if (rc) return rc;
  const sdp_split_args rd = with_readable_demands(args);
  const sdp_split_args* fwd = &rd;
  if (!fwd->dist) return fail(SDP_ERR_UNSUPPORTED, "the adjoint is taken with respect to dist: set dist, not coords");
  if (fwd->capacity_mode != SDP_CAPACITY_HARD)
    return fail(SDP_ERR_UNSUPPORTED, "the adjoint takes the hard capacity only");
  if (!is_device_ptr(grad_mean)) return fail(SDP_ERR_INVALID_ARG, "grad_mean must be a device pointer");
  if (!is_device_ptr(grad_dist)) return fail(SDP_ERR_INVALID_ARG, "grad_dist must be a device pointer");
  if (route_hist_out && !is_device_ptr(route_hist_out))
    return fail(SDP_ERR_INVALID_ARG, "route_hist_out must be a device pointer");
  if (pred && !is_device_ptr(pred)) return fail(SDP_ERR_INVALID_ARG, "pred must be a device pointer");
  if (pred && fwd->pred_dtype != SDP_PRED_U16 && fwd->pred_dtype != SDP_PRED_I32)
    return fail(SDP_ERR_INVALID_ARG, "pred_dtype must be SDP_PRED_U16 or SDP_PRED_I32");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SplitWs need = carve_split(fwd, nullptr, true);
  rc = check_ws(fwd->workspace, fwd->workspace_bytes, need.bytes);
  if (rc) return rc;
  uint32_t* status;
  rc = status_ptr(&status);
  if (rc) return rc;
  rc = fault_call();
  if (rc) return rc;
  const SplitWs w = carve_split(fwd, fwd->workspace, true);
  const int n = fwd->n;
  cudaError_t e = cudaMemsetAsync(w.hist, 0, sizeof(unsigned long long) * (2 * (size_t)n + 1), st);
  if (e != cudaSuccess) return cuda_fail(e, "memset hist");
  if (n > 0 && fwd->S > 0) {
    if (pred) {
      launch_backtrack_hist(n, fwd->S, pred, fwd->pred_dtype, w.hist, status, st);
    } else {
      launch_tour_prep(fwd->tour, n, fwd->coords, fwd->dist, w.prep, status, w.fb_count, st);
      rc = run_split_core(fwd, w, status, w.hist, st);
      if (rc) return rc;
    }
  }
  launch_grad_assemble(n, fwd->S, fwd->tour, w.hist, grad_mean, grad_dist, route_hist_out, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return SDP_OK;
}

namespace {
// the lane kernel keeps its decision bits in the workspace when the policy
// is wanted
bool reinsert_uses_lane(const sdp_reinsert_args* a) {
  return (a->algo == SDP_REINSERT_LANE || a->algo == SDP_REINSERT_AUTO) &&
         !(a->n_routes > 0 && a->end_cost_table) &&
         reinsert_lane_supported(a->T, a->U, a->n_routes);
}
size_t reinsert_scratch_bytes(const sdp_reinsert_args* a) {
  return (reinsert_uses_lane(a) && a->policy_out && a->S > 0)
             ? reinsert_lane_scratch_bytes(a->T, a->U) : 0;
}
}  // namespace

size_t sdp_reinsert_workspace_bytes(const sdp_reinsert_args* a) {
  if (!a || a->S < 0 || a->T < 1 || a->U < 0) return 0;
  return align_up((size_t)kMeanBlocks * sizeof(double), 256) + reinsert_scratch_bytes(a);
}

int sdp_reinsert_eval(const sdp_reinsert_args* a, void* stream) {
  if (!a) return fail(SDP_ERR_INVALID_ARG, "args is NULL");
  if (a->T < 1 || a->T > 4096) return fail(SDP_ERR_INVALID_ARG, "T = %d outside 1..4096", a->T);
  if (a->U < 0 || a->U > 1023) return fail(SDP_ERR_INVALID_ARG, "U = %d outside 0..1023", a->U);
  if (a->I0 < 0 || a->I0 > a->U) return fail(SDP_ERR_INVALID_ARG, "I0 = %d outside 0..U", a->I0);
  if (a->S < 0) return fail(SDP_ERR_INVALID_ARG, "S < 0");
  if (a->algo < SDP_REINSERT_AUTO || a->algo > SDP_REINSERT_LANE)
    return fail(SDP_ERR_INVALID_ARG, "unknown reinsertion algo %d", a->algo);
  if (a->n_routes < 0 || a->n_routes > 64)
    return fail(SDP_ERR_INVALID_ARG, "n_routes = %d outside 0..64", a->n_routes);
  if (a->n_routes > 0) {
    if (a->U > 255) return fail(SDP_ERR_UNSUPPORTED, "route options need U <= 255");
    if (a->end_cost_table) return fail(SDP_ERR_UNSUPPORTED, "route options take linear end costs");
    if (a->S > 0 && (!is_device_ptr(a->route_cost) || !is_device_ptr(a->route_cap)))
      return fail(SDP_ERR_INVALID_ARG, "route_cost / route_cap must be device pointers");
  }
  if (a->algo == SDP_REINSERT_LANE && !reinsert_lane_supported(a->T, a->U, a->n_routes))
    return fail(SDP_ERR_UNSUPPORTED,
                "SDP_REINSERT_LANE needs U <= 255, at most 8 route options and its shared memory to fit");
  const int kc = a->U + 1 <= 256 ? (a->U + 1 + 31) / 32 : (a->U + 1 <= 512 ? 16 : 32);
  const int64_t words = (int64_t)a->T * ((kc + 7) & ~7);
  if (words > 4096)
    return fail(SDP_ERR_UNSUPPORTED,
                "T = %d with U = %d needs %lld decision words per scenario, above 4096 "
                "(decision bits are kept on chip)", a->T, a->U, (long long)words);
  if (a->S > 0) {
    if (a->n_routes == 0 && !is_device_ptr(a->fixed))
      return fail(SDP_ERR_INVALID_ARG, "fixed must be a device pointer");
    if (!is_device_ptr(a->consumption)) return fail(SDP_ERR_INVALID_ARG, "consumption must be a device pointer");
    if (!is_device_ptr(a->value_out)) return fail(SDP_ERR_INVALID_ARG, "value_out must be a device pointer");
    if (a->end_cost_table && !is_device_ptr(a->end_cost_table))
      return fail(SDP_ERR_INVALID_ARG, "end_cost_table must be a device pointer");
    if (a->policy_out && !is_device_ptr(a->policy_out))
      return fail(SDP_ERR_INVALID_ARG, "policy_out must be a device pointer");
    if (a->value0_out && !is_device_ptr(a->value0_out))
      return fail(SDP_ERR_INVALID_ARG, "value0_out must be a device pointer");
  }
  if (a->mean_out && !is_device_ptr(a->mean_out)) return fail(SDP_ERR_INVALID_ARG, "mean_out must be a device pointer");
  const size_t need = sdp_reinsert_workspace_bytes(a);
  const size_t scratch = reinsert_scratch_bytes(a);
  int rc = (a->mean_out || scratch) ? check_ws(a->workspace, a->workspace_bytes, need) : SDP_OK;
  if (rc) return rc;
  uint32_t* status;
  rc = status_ptr(&status);
  if (rc) return rc;
  rc = fault_call();
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ReinsertArgs r{};
  r.algo = a->algo; r.T = a->T; r.U = a->U; r.I0 = a->I0;
  r.n_routes = a->n_routes; r.route_cost = a->route_cost; r.route_cap = a->route_cap; r.h = a->h; r.p = a->p; r.c = a->unit_cost;
  r.S = a->S; r.fixed = a->fixed; r.table = a->end_cost_table; r.cons = a->consumption;
  r.value = a->value_out; r.policy = a->policy_out; r.value0 = a->value0_out; r.status = status;
  r.dscratch = scratch ? reinterpret_cast<uint32_t*>(
                             static_cast<unsigned char*>(a->workspace) +
                             align_up((size_t)kMeanBlocks * sizeof(double), 256))
                       : nullptr;
  prof_begin(st);
  int e = launch_reinsert(r, st);
  prof_end(st);
  if (e) return cuda_fail((cudaError_t)e, "reinsert launch");
  if (a->mean_out) {
    launch_mean(a->value_out, a->S, static_cast<double*>(a->workspace), a->mean_out, st);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "mean launch");
  }
  return SDP_OK;
}

}  // extern "C"
