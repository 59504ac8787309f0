// split_batch.cu -- plans for batched Split: thousands of giant tours of
// uneven length (first-stage candidates) times S scenarios each, evaluated by
// one persistent launch replayed from a CUDA graph.
//
// A plan owns: per-tour metadata on the device (n_b, offsets, the order of
// tours by decreasing n_b), the concatenated tour records, the per-tour D(n)
// in FP64, the work-queue counter, the fallback list and its scratch.  One
// run = [tour prep for every tour (also resets the counter) -> persistent
// kernel over (tour, 32-scenario tile) items -> recomputation of the
// scenarios it flagged (one warp each, split_rescue.cu, where the longest
// tour fits its shared memory; else the plain per-scenario kernel) ->
// per-tour FP64 means], captured once in a CUDA graph and replayed.  The persistent kernel is the pipelined one
// (split_pipe_kernel: producer warps narrow each tile's rows into tour order
// in an L2-resident slot ring, 23 DP warps per SM) when the demand offsets
// allow bulk copies and every tour has n <= 1024, else the streaming one
// (split_batch_stream_kernel), else the DEQUE batched kernel.
// sdp_plan_autotune times the launch shapes (pipelined; streaming; DEQUE
// warps per CTA x deque ring size) and keeps the fastest; choices can be
// cached in a text file keyed by the device and the plan's shape.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "sdp_internal.cuh"

struct sdp_plan {
  int device = 0;
  int B = 0, Q = 0, n_max = 0;
  int64_t S = 0, sum_n = 0;
  // device arrays owned by the plan
  int32_t* d_n = nullptr;
  int64_t* d_tour_off = nullptr;
  int64_t* d_coord_off = nullptr;
  int64_t* d_dem_off = nullptr;
  int64_t* d_rec_off = nullptr;
  int32_t* d_order = nullptr;
  sdp::StepRec* d_rec = nullptr;
  double* d_Dn = nullptr;
  unsigned long long* d_counter = nullptr;
  uint32_t* d_fb_count = nullptr;
  unsigned long long* d_fb_list = nullptr;
  float* d_kscratch = nullptr;
  int64_t nslots = 0;
  unsigned long long* d_total = nullptr;
  unsigned char* d_qt = nullptr;  // row slots of the streaming kernel, or NULL
  unsigned char* d_pq = nullptr;  // slot ring of the pipelined kernel, or NULL
  // caller's arrays
  const int32_t* tours = nullptr;
  const float* coords = nullptr;
  const int32_t* demands = nullptr;
  float* costs = nullptr;
  double* means = nullptr;
  // launch shape; warps == -1: the streaming kernel, -2: the pipelined one;
  // ns: scenarios per lane (DEQUE kernel with shared-memory staging)
  int warps = 4, ring = 16, ns = 1, grid = 0;
  // graph
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the persistent kernel
  int64_t total_arcs = -1;
};

namespace sdp {
int status_word(uint32_t** out);               // sdp_api.cu
int api_fail(int code, const char* msg);       // sdp_api.cu
namespace {

int pfail(int code, const char* msg) { return api_fail(code, msg); }

int pcuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return api_fail(SDP_ERR_CUDA, buf);
}

template <typename T>
cudaError_t alloc_copy(T** dst, const T* src, size_t count) {
  if (fault_alloc()) return cudaErrorMemoryAllocation;  // injected (tests)
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) return e;
  if (src && count) e = cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
  return e;
}

BatchPrepArgs prep_args(const sdp_plan* p, uint32_t* status) {
  BatchPrepArgs a{};
  a.n = p->d_n;
  a.tour_off = p->d_tour_off;
  a.coord_off = p->d_coord_off;
  a.rec_off = p->d_rec_off;
  a.tours = p->tours;
  a.coords = p->coords;
  a.rec = p->d_rec;
  a.Dn = p->d_Dn;
  a.counter = p->d_counter;
  a.fb_count = p->d_fb_count;
  a.status = status;
  return a;
}

int configure(sdp_plan* p, int warps, int ring, int ns = 1) {
  if (ns != 1 && ns != 2) return SDP_ERR_UNSUPPORTED;
  if (ns == 2 && warps <= 0) return SDP_ERR_UNSUPPORTED;  // shared-memory DEQUE only
  if (ring != 8 && ring != 16 && ring != 32) return SDP_ERR_UNSUPPORTED;
  if (warps == -2) {  // pipelined kernel: one CTA per SM, ring of 16 entries
    if (!p->d_pq) return SDP_ERR_UNSUPPORTED;
    p->warps = -2;
    p->ring = 16;
    p->ns = 1;
    p->grid = pipe_grid(p->S, p->B, true);
    return SDP_OK;
  }
  if (warps < 0) {  // streaming kernel: one CTA per SM, ring of 16 entries
    if (!p->d_qt) return SDP_ERR_UNSUPPORTED;
    p->warps = -1;
    p->ring = 16;
    p->ns = 1;
    p->grid = num_sms();
    return SDP_OK;
  }
  if (warps > 8) return SDP_ERR_UNSUPPORTED;
  if (batch_smem(p->n_max, p->Q, warps, ring, ns) > 227 * 1024) return SDP_ERR_UNSUPPORTED;
  BatchKernelArgs k{};
  k.n_max = p->n_max;
  k.Q = p->Q;
  int occ = 0;
  int e = launch_split_batch(k, warps, ring, ns, 0, nullptr, &occ);
  if (e) return pcuda((cudaError_t)e, "batch occupancy");
  if (occ < 1) return SDP_ERR_UNSUPPORTED;
  const int64_t items = (int64_t)p->B * ((((p->S + 31) / 32) + ns - 1) / ns);
  const int eff = warps > 0 ? warps : batch_tmem_warps(p->n_max, p->Q);
  const int64_t want = (items + eff - 1) / eff;
  p->warps = warps;
  p->ring = ring;
  p->ns = ns;
  p->grid = (int)std::min<int64_t>(want, (int64_t)occ * num_sms());
  return SDP_OK;
}

int enqueue(sdp_plan* p, cudaStream_t st, uint32_t* status, bool with_events) {
  launch_batch_prep(prep_args(p, status), p->B, st);
  BatchKernelArgs k{};
  k.B = p->B; k.Q = p->Q; k.n_max = p->n_max; k.S = p->S;
  k.n = p->d_n; k.dem_off = p->d_dem_off; k.rec_off = p->d_rec_off; k.order = p->d_order;
  k.rec = p->d_rec; k.Dn = p->d_Dn; k.demands = p->demands; k.costs = p->costs;
  k.counter = p->d_counter; k.fb_list = p->d_fb_list; k.fb_count = p->d_fb_count;
  k.status = status;
  // External records become event-record nodes of the captured graph (a plain
  // record inside a capture only orders streams and never fires).
  if (with_events) cudaEventRecordWithFlags(p->ev0, st, cudaEventRecordExternal);
  int e;
  if (p->warps == -2) {
    PipeArgs pa{};
    pa.batched = 1;
    pa.B = p->B; pa.Q = p->Q; pa.S = p->S;
    pa.n = p->d_n; pa.dem_off = p->d_dem_off; pa.rec_off = p->d_rec_off; pa.order = p->d_order;
    pa.rec = p->d_rec; pa.Dn = p->d_Dn; pa.demands = p->demands; pa.cost = p->costs;
    pa.qt = p->d_pq; pa.stride = pipe_row_stride(p->n_max, p->Q); pa.counter = p->d_counter;
    pa.n_max = p->n_max;
    pa.fb_count = p->d_fb_count; pa.fb_list = p->d_fb_list; pa.status = status;
    e = launch_split_pipe(pa, st);
  } else if (p->warps < 0) {
    BatchStreamArgs sa{};
    sa.B = p->B; sa.Q = p->Q; sa.S = p->S;
    sa.n = p->d_n; sa.dem_off = p->d_dem_off; sa.rec_off = p->d_rec_off; sa.order = p->d_order;
    sa.rec = p->d_rec; sa.Dn = p->d_Dn; sa.demands = p->demands; sa.costs = p->costs;
    sa.counter = p->d_counter; sa.fb_list = p->d_fb_list; sa.fb_count = p->d_fb_count;
    sa.status = status; sa.qt = p->d_qt; sa.stride_max = batch_stream_stride(p->n_max, p->Q);
    e = launch_split_batch_stream(sa, st);
  } else {
    e = launch_split_batch(k, p->warps, p->ring, p->ns, p->grid, st, nullptr);
  }
  if (with_events) cudaEventRecordWithFlags(p->ev1, st, cudaEventRecordExternal);
  if (e) return pcuda((cudaError_t)e, "batch kernel");
  if (rescue_supported(p->n_max)) {
    // the entries the DP kernel flagged, one warp each
    RescueArgs r{};
    r.batched = 1; r.Q = p->Q; r.S = p->S; r.n_max = p->n_max;
    r.n = p->d_n; r.rec_off = p->d_rec_off; r.dem_off = p->d_dem_off;
    r.fb_list = p->d_fb_list; r.costs = p->costs;
    r.rec = p->d_rec; r.Dn = p->d_Dn; r.demands = p->demands;
    r.fb_count = p->d_fb_count; r.status = status;
    const int er = launch_split_rescue(r, (int64_t)p->B * p->S, st);
    if (er) return pcuda((cudaError_t)er, "batch rescue");
  } else {
    BatchFallbackArgs f{};
    f.Q = p->Q; f.S = p->S; f.n = p->d_n; f.dem_off = p->d_dem_off; f.rec_off = p->d_rec_off;
    f.rec = p->d_rec; f.Dn = p->d_Dn; f.demands = p->demands; f.costs = p->costs;
    f.fb_list = p->d_fb_list; f.fb_count = p->d_fb_count; f.kscratch = p->d_kscratch;
    f.nslots = p->nslots;
    launch_batch_fallback(f, st);
  }
  if (p->means) launch_batch_means(p->costs, p->B, p->S, p->means, st);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return pcuda(ce, "batch enqueue");
  return SDP_OK;
}

void drop_graph(sdp_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
}

std::string cache_key(const sdp_plan* p) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, p->device);
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|sm%d|B%d|S%lld|Q%d|nmax%d|sumn%lld", prop.name,
           prop.multiProcessorCount, p->B, (long long)p->S, p->Q, p->n_max,
           (long long)p->sum_n);
  std::string k(buf);
  for (char& c : k)
    if (c == ' ') c = '_';
  return k;
}

}  // namespace
}  // namespace sdp

using namespace sdp;

extern "C" {

void sdp_plan_destroy(sdp_plan* p) {
  if (!p) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  drop_graph(p);
  cudaFree(p->d_n); cudaFree(p->d_tour_off); cudaFree(p->d_coord_off);
  cudaFree(p->d_dem_off); cudaFree(p->d_rec_off); cudaFree(p->d_order);
  cudaFree(p->d_rec); cudaFree(p->d_Dn); cudaFree(p->d_counter); cudaFree(p->d_fb_count);
  cudaFree(p->d_fb_list); cudaFree(p->d_kscratch); cudaFree(p->d_total); cudaFree(p->d_qt);
  cudaFree(p->d_pq);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  cudaSetDevice(prev);
  delete p;
}

int sdp_split_plan_create(const sdp_split_batch_desc* d, sdp_plan** out) {
  if (!d || !out) return pfail(SDP_ERR_INVALID_ARG, "desc / out is NULL");
  *out = nullptr;
  if (d->B < 1) return pfail(SDP_ERR_INVALID_ARG, "B < 1");
  if (d->Q < 1 || d->Q > 32767) return pfail(SDP_ERR_UNSUPPORTED, "batched Split needs 1 <= Q <= 32767");
  if (d->S < 1) return pfail(SDP_ERR_INVALID_ARG, "S < 1");
  if ((double)d->B * (double)d->S > 1.8e19) return pfail(SDP_ERR_UNSUPPORTED, "B*S too large");
  if (!d->n_host || !d->tour_off_host || !d->coord_off_host || !d->dem_off_host)
    return pfail(SDP_ERR_INVALID_ARG, "host offset arrays must be set");
  if (!d->tours || !d->coords || !d->demands || !d->costs_out)
    return pfail(SDP_ERR_INVALID_ARG, "tours / coords / demands / costs_out must be set");
  auto* p = new sdp_plan();
  cudaGetDevice(&p->device);
  p->B = d->B; p->Q = d->Q; p->S = d->S;
  p->tours = d->tours; p->coords = d->coords; p->demands = d->demands;
  p->costs = d->costs_out; p->means = d->means_out;
  std::vector<int64_t> rec_off(d->B);
  for (int b = 0; b < d->B; ++b) {
    const int n = d->n_host[b];
    if (n < 1 || n > 65534) { sdp_plan_destroy(p); return pfail(SDP_ERR_UNSUPPORTED, "n_b outside 1..65534"); }
    if (d->tour_off_host[b] < 0 || d->coord_off_host[b] < 0 || d->dem_off_host[b] < 0) {
      sdp_plan_destroy(p);
      return pfail(SDP_ERR_INVALID_ARG, "negative offset");
    }
    rec_off[b] = p->sum_n;
    p->sum_n += n;
    p->n_max = std::max(p->n_max, n);
  }
  std::vector<int32_t> order(d->B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return d->n_host[a] > d->n_host[b]; });
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chk(alloc_copy(&p->d_n, d->n_host, d->B));
  chk(alloc_copy(&p->d_tour_off, d->tour_off_host, d->B));
  chk(alloc_copy(&p->d_coord_off, d->coord_off_host, d->B));
  chk(alloc_copy(&p->d_dem_off, d->dem_off_host, d->B));
  chk(alloc_copy(&p->d_rec_off, rec_off.data(), d->B));
  chk(alloc_copy(&p->d_order, order.data(), d->B));
  chk(alloc_copy<StepRec>(&p->d_rec, nullptr, p->sum_n));
  chk(alloc_copy<double>(&p->d_Dn, nullptr, d->B));
  chk(alloc_copy<unsigned long long>(&p->d_counter, nullptr, 1));
  chk(alloc_copy<uint32_t>(&p->d_fb_count, nullptr, 1));
  chk(alloc_copy<unsigned long long>(&p->d_fb_list, nullptr, (size_t)d->B * d->S));
  p->nslots = std::min<int64_t>((int64_t)d->B * d->S, 4096);
  chk(alloc_copy<float>(&p->d_kscratch, nullptr, (size_t)(p->n_max + 1) * p->nslots));
  chk(alloc_copy<unsigned long long>(&p->d_total, nullptr, 1));
  // the streaming kernel bulk-copies each tile's rows: they must start on
  // 16 bytes (element offsets that are multiples of 4, an aligned base)
  bool stream_ok = batch_stream_supported(p->n_max, p->Q) &&
                   (reinterpret_cast<uintptr_t>(d->demands) & 15) == 0;
  for (int b = 0; stream_ok && b < d->B; ++b) stream_ok = (d->dem_off_host[b] & 3) == 0;
  if (stream_ok) chk(alloc_copy<unsigned char>(&p->d_qt, nullptr, batch_stream_qt_bytes(p->n_max, p->Q)));
  // the pipelined kernel bulk-copies the same way, for tours of n <= 1024
  if (stream_ok && pipe_supported(p->n_max, p->Q))
    chk(alloc_copy<unsigned char>(&p->d_pq, nullptr,
                                  pipe_ring_bytes(p->n_max, p->Q, p->S, p->B, true)));
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sdp_plan_destroy(p);
    return e == cudaErrorMemoryAllocation ? pfail(SDP_ERR_OOM, "plan allocation failed")
                                          : pcuda(e, "plan create");
  }
  int rc = configure(p, -2, 16);  // pipelined kernel when the plan allows it
  if (rc == SDP_ERR_UNSUPPORTED) rc = configure(p, -1, 16);  // else the streaming one
  if (rc == SDP_ERR_UNSUPPORTED) rc = configure(p, 0, 16);  // TMEM staging when the tours fit
  if (rc == SDP_ERR_UNSUPPORTED) rc = configure(p, 4, 16);
  if (rc == SDP_ERR_UNSUPPORTED) rc = configure(p, 1, 8);
  if (rc) {
    sdp_plan_destroy(p);
    return pfail(rc, "no launch shape of the batched kernel fits this plan");
  }
  *out = p;
  return SDP_OK;
}

int sdp_plan_run(sdp_plan* p, void* stream) {
  if (!p) return pfail(SDP_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status;
  int rc = status_word(&status);
  if (rc) return rc;
  rc = fault_call_hook();
  if (rc) return rc;
  if (!p->exec) {
    // capture on a private stream so the caller's stream may be the legacy one
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return pcuda(e, "capture stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return pcuda(e, "begin capture"); }
    rc = enqueue(p, cs, status, true);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return pcuda(e, "end capture");
    e = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { p->exec = nullptr; return pcuda(e, "graph instantiate"); }
  }
  cudaError_t e = cudaGraphLaunch(p->exec, st);
  if (e != cudaSuccess) return pcuda(e, "graph launch");
  return SDP_OK;
}

int sdp_plan_kernel_ms(sdp_plan* p, float* ms) {
  if (!p || !ms) return pfail(SDP_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaEventSynchronize(p->ev1);
  if (e != cudaSuccess) return pcuda(e, "event sync");
  e = cudaEventElapsedTime(ms, p->ev0, p->ev1);
  if (e != cudaSuccess) return pcuda(e, "elapsed");
  return SDP_OK;
}

int sdp_plan_info(const sdp_plan* p, int32_t* warps_per_cta, int32_t* ring, int32_t* ctas,
                  int64_t* items) {
  if (!p) return pfail(SDP_ERR_INVALID_ARG, "plan is NULL");
  if (warps_per_cta) *warps_per_cta = p->warps;
  if (ring) *ring = p->ring;
  if (ctas) *ctas = p->grid;
  if (items) *items = (int64_t)p->B * ((p->S + 31) / 32);
  return SDP_OK;
}

}  // extern "C"

namespace sdp {
// min_ring: the smallest deque ring timed.  Plans whose tours change between
// runs (the SAA search) take 16: a ring sized on the tours it was timed on can
// overflow on later ones, and every overflowed scenario is recomputed.
int plan_autotune(sdp_plan* p, void* stream, const char* cache_path, int min_ring) {
  if (!p) return pfail(SDP_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::string key = cache_key(p);
  if (min_ring > 8) key += "|ring>=" + std::to_string(min_ring);
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[512];
      while (fgets(line, sizeof(line), f)) {
        char k[400];
        int w = 0, r = 0, ns = 1;
        const int got = sscanf(line, "%399s %d %d %d", k, &w, &r, &ns);
        if (got >= 3 && key == k) {
          fclose(f);
          drop_graph(p);
          int rc = configure(p, w, r, got == 4 ? ns : 1);
          return rc ? configure(p, 1, 8) : SDP_OK;  // cached shape no longer fits
        }
      }
      fclose(f);
    }
  }
  uint32_t* status;
  int rc = status_word(&status);
  if (rc) return rc;
  const int warps_c[] = {-2, -1, 0, 1, 2, 4, 8};  // -2 pipelined, -1 streaming, 0 TMEM staging
  const int ring_c[] = {8, 16};
  const int ns_c[] = {1, 2};  // scenarios per lane (shared-memory staging only)
  float best = 1e30f;
  int bw = p->warps, br = p->ring, bn = p->ns;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int w : warps_c)
    for (int r : ring_c)
    for (int ns : ns_c) {
      if (w < 0 && r != 16) continue;  // the pipelined / streaming kernels have one ring size
      if (w <= 0 && ns != 1) continue;
      if (r < min_ring) continue;
      if (configure(p, w, r, ns)) continue;
      float tsum = 0.f;
      bool ok = true;
      for (int rep = 0; rep < 3 && ok; ++rep) {
        cudaEventRecord(a, st);
        ok = enqueue(p, st, status, false) == SDP_OK;
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) tsum += ms;  // first rep warms up
      }
      if (ok && tsum < best) { best = tsum; bw = w; br = r; bn = ns; }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  drop_graph(p);
  rc = configure(p, bw, br, bn);
  if (rc) return rc;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "%s %d %d %d\n", key.c_str(), bw, br, bn);
      fclose(f);
    }
  }
  return SDP_OK;
}
}  // namespace sdp

extern "C" {

int sdp_plan_autotune(sdp_plan* p, void* stream, const char* cache_path) {
  return plan_autotune(p, stream, cache_path, 8);
}

int sdp_plan_configure(sdp_plan* p, int32_t warps_per_cta, int32_t ring, int32_t scenarios_per_lane) {
  if (!p) return pfail(SDP_ERR_INVALID_ARG, "plan is NULL");
  const int old_w = p->warps, old_r = p->ring, old_n = p->ns;
  const int rc = configure(p, warps_per_cta, ring, scenarios_per_lane);
  if (rc) {
    configure(p, old_w, old_r, old_n);  // keep the plan usable
    return rc == SDP_ERR_UNSUPPORTED ? pfail(rc, "launch shape not available for this plan") : rc;
  }
  drop_graph(p);
  return SDP_OK;
}

int sdp_plan_scenarios_per_lane(const sdp_plan* p, int32_t* ns) {
  if (!p || !ns) return pfail(SDP_ERR_INVALID_ARG, "NULL argument");
  *ns = p->ns;
  return SDP_OK;
}

int sdp_plan_count_arcs(sdp_plan* p, void* stream, uint64_t* total_host) {
  if (!p || !total_host) return pfail(SDP_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status;
  int rc = status_word(&status);
  if (rc) return rc;
  cudaMemsetAsync(p->d_total, 0, sizeof(unsigned long long), st);
  launch_batch_prep(prep_args(p, status), p->B, st);
  launch_batch_count(prep_args(p, status), p->B, p->S, p->Q, p->d_dem_off, p->demands,
                     p->d_total, st);
  unsigned long long t = 0;
  cudaError_t e = cudaMemcpyAsync(&t, p->d_total, sizeof(t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return pcuda(e, "count arcs");
  *total_host = t;
  p->total_arcs = (int64_t)t;
  return SDP_OK;
}

}  // extern "C"
