// batch.cu -- several lattices of uneven size (SU(2) and SU(3) fundamental,
// each with its own number of right-hand sides) in one persistent launch.
//
// The host turns the batch into a task table, passed to the kernel by value
// as a launch parameter (no host-to-device copy, so a launch can be captured
// into a CUDA graph): one task per (lattice, output parity, phase), each
// covering V_h * n_rhs thread slots cut into chunks of one block.  Blocks of a cooperative grid (every block
// resident) take chunks from a device work queue (an atomic counter per
// phase), so small and large lattices share the GPU without one launch per
// lattice.  The full operator D needs one phase; the even-odd operator
// Dhat = A - H_eo H_oe / (4A) needs two (the odd temporaries of phase 0 feed
// phase 1), separated by a grid barrier.  The barrier wait is bounded by the
// global timer: a block that waits longer than the limit raises an error flag
// and returns, and the call reports BSM_ETIMEOUT instead of hanging.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <mutex>
#include <string>
#include <vector>

#include "batch.cuh"
#include "mrhs.cuh"
#include "operators.cuh"

namespace bsm {

namespace {

struct BatchTask {
  MrhsArgs args;       // geometry, links of the output parity, in / out / x, a, b, nrhs
  int d;               // 2 or 3
  int phase;
  long long chunk0;    // first chunk of this task within its phase
  long long chunks;
};

constexpr int kMaxPhases = 4;

struct BatchControl {
  unsigned long long next[kMaxPhases];  // work-queue counters, one per phase
  unsigned int arrived;                 // block arrivals at the grid barriers so far
  int error;                            // 1: a barrier wait timed out
};

struct BatchMeta {
  int ntasks;
  int nphases;
  int grab;                       // chunks taken per work-queue grab
  long long phase_chunks[kMaxPhases];
  unsigned int grid_blocks;       // the barrier after phase j waits for (j + 1) * grid_blocks + barrier_extra arrivals
  unsigned int barrier_extra;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kMaxBatchTasks = 128;    // up to 4 tasks per lattice (Dhat^+ Dhat), 32 lattices per launch
// launch configuration: RHS per thread (RB) and chunks per work-queue grab;
// picked per batch shape by timing (batch_tuned_config), or the default
struct BatchConfig {
  int rb = 1;           // RHS per thread: 1 or 2, or 2 and 4 as packed pairs
  int grab = 4;
  bool paired = false;  // RHS held two per f32x2 register pair (bit-identical results)
};

// the whole task table as one launch parameter (the parameter space holds up
// to 32 KB from CUDA 12.1 on sm_70+)
struct BatchTable {
  BatchTask t[kMaxBatchTasks];
};
static_assert(sizeof(BatchTable) + sizeof(BatchMeta) + sizeof(void*) < 32000, "batch table exceeds the parameter space");

// RB = 1: 128 registers, 4 blocks per SM (measured: 7 % faster than 168 / 3
// on the 16-lattice batch, as for the d = 3 multi-RHS kernel); RB = 2: two
// RHS per thread (each link element applied to both), 2 blocks per SM;
// PAIRED: RB = 2 or 4 RHS per thread as lane pairs of packed FP32
// instructions (the multi-RHS paired kernel's site code).  A thread slot of
// a task is (site, block of RB RHS).
template <int RB, bool PAIRED>
__global__ void __launch_bounds__(kHopThreads, RB == 1 ? 4 : 2) batch_kernel(const __grid_constant__ BatchTable table,
                                                                             BatchControl* ctl, const BatchMeta meta) {
  __shared__ BatchTask s_tasks[kMaxBatchTasks];
  __shared__ long long s_chunk;
  __shared__ int s_abort;
  for (int k = threadIdx.x; k < meta.ntasks; k += kHopThreads) s_tasks[k] = table.t[k];
  __syncthreads();
  for (int phase = 0; phase < meta.nphases; ++phase) {
    // this phase's tasks occupy a contiguous range of the table
    int first = 0;
    while (first < meta.ntasks && s_tasks[first].phase != phase) ++first;
    for (;;) {
      if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(&ctl->next[phase], 1ull) * meta.grab;
      __syncthreads();
      const long long c0 = s_chunk;
      __syncthreads();
      if (c0 >= meta.phase_chunks[phase]) break;
      int k = first;
      for (int sub = 0; sub < meta.grab; ++sub) {
        const long long c = c0 + sub;
        if (c >= meta.phase_chunks[phase]) break;
        while (c >= s_tasks[k].chunk0 + s_tasks[k].chunks) ++k;  // chunks ascend with k
        const BatchTask& tk = s_tasks[k];
        const long long u = (c - tk.chunk0) * kHopThreads + threadIdx.x;
        const int nblk = tk.args.nrhs / RB;
        if (u < (long long)tk.args.g.Vh * nblk) {
          const int i = (int)(u / nblk), r = (int)(u - (long long)i * nblk) * RB;
          // later phases read what an earlier phase of this launch wrote: through L2 only
          if constexpr (PAIRED) {
            if (phase == 0) {
              if (tk.d == 2) mrhs_site_paired<F32, 2, false, RB / 2>(tk.args, i, r);
              else mrhs_site_paired<F32, 3, false, RB / 2>(tk.args, i, r);
            } else {
              if (tk.d == 2) mrhs_site_paired<F32, 2, false, RB / 2, true>(tk.args, i, r);
              else mrhs_site_paired<F32, 3, false, RB / 2, true>(tk.args, i, r);
            }
          } else if (phase == 0) {
            if (tk.d == 2) mrhs_site<F32, 2, false, RB>(tk.args, i, r);
            else mrhs_site<F32, 3, false, RB>(tk.args, i, r);
          } else {
            if (tk.d == 2) mrhs_site<F32, 2, false, RB, true>(tk.args, i, r);
            else mrhs_site<F32, 3, false, RB, true>(tk.args, i, r);
          }
        }
      }
    }
    if (phase + 1 < meta.nphases) {
      // grid barrier: every block of the cooperative grid arrives once per
      // barrier, after all its threads have made their phase writes visible
      // device-wide
      const unsigned target = (unsigned)(phase + 1) * meta.grid_blocks + meta.barrier_extra;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->arrived, 1u);
        const unsigned long long t0 = global_ns();
        int abort = 0;
        // two independent bounds: the global timer and an iteration count
        // (2^24 polls of >= 256 ns), so the wait ends even if the timer stalls
        for (unsigned it = 0; *(volatile unsigned int*)&ctl->arrived < target; ++it) {
          if (*(volatile int*)&ctl->error != 0 || global_ns() - t0 > meta.timeout_ns || it > (1u << 24)) {
            atomicExch(&ctl->error, 1);
            abort = 1;
            break;
          }
          __nanosleep(256);
        }
        __threadfence();
        s_abort = abort;
      }
      __syncthreads();
      if (s_abort) return;
    }
  }
}

BatchTask with_tasks_scalars(BatchTask t) {
  t.args = with_f32_scalars(t.args);
  return t;
}

}  // namespace

namespace {

// the tasks (ordered by phase) as one cooperative launch: chunk offsets,
// grid size (every block resident, so that the grid barriers complete),
// the control block reset, the launch
int launch_tasks(std::vector<BatchTask> tasks, BatchMeta meta, BatchControl* ctl, double timeout_s,
                 int barrier_extra, const BatchConfig& cfg, cudaStream_t s) {
  if ((int)tasks.size() > kMaxBatchTasks) return BSM_EUNSUPPORTED;
  // The queue hands out chunks in table order: within a phase, the d = 3
  // tasks before the d = 2 ones (so that the blocks run one site routine at a
  // time, not both), and large tasks before small ones (the small ones fill
  // the tail).  Each task writes only its own output, so the order changes
  // no result.
  std::stable_sort(tasks.begin(), tasks.end(), [](const BatchTask& a, const BatchTask& b) {
    if (a.phase != b.phase) return a.phase < b.phase;
    if (a.d != b.d) return a.d > b.d;
    return a.chunks > b.chunks;
  });
  for (int ph = 0; ph < meta.nphases; ++ph) meta.phase_chunks[ph] = 0;
  for (BatchTask& t : tasks) {
    t.chunk0 = meta.phase_chunks[t.phase];
    meta.phase_chunks[t.phase] += t.chunks;
  }
  meta.ntasks = (int)tasks.size();
  meta.grab = cfg.grab;
  const void* kern = cfg.paired ? (cfg.rb == 4 ? (const void*)batch_kernel<4, true> : (const void*)batch_kernel<2, true>)
                                : (cfg.rb == 2 ? (const void*)batch_kernel<2, false> : (const void*)batch_kernel<1, false>);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHopThreads, 0) != cudaSuccess || per_sm < 1)
    return BSM_ECUDA;
  long long want = 0;
  for (int ph = 0; ph < meta.nphases; ++ph) want = meta.phase_chunks[ph] > want ? meta.phase_chunks[ph] : want;
  want = (want + cfg.grab - 1) / cfg.grab;
  int grid = sms * per_sm;
  if (want < grid) grid = (int)(want > 0 ? want : 1);
  meta.grid_blocks = (unsigned)grid;
  meta.barrier_extra = (unsigned)(barrier_extra > 0 ? barrier_extra : 0);
  meta.timeout_ns = (unsigned long long)((timeout_s > 0 ? timeout_s : 1.0) * 1e9);

  BatchTable table;
  memset(&table, 0, sizeof(table));
  for (size_t k = 0; k < tasks.size(); ++k) table.t[k] = tasks[k];
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(BatchControl), s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  void* kargs[] = {(void*)&table, (void*)&ctl, (void*)&meta};
  e = cudaLaunchCooperativeKernel(kern, grid, kHopThreads, kargs, 0, s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return BSM_OK;
}

}  // namespace

// validated by the caller: SU(2)/SU(3) fundamental, FP32, nrhs >= 1
size_t batch_workspace_bytes(const bsm_batch_item* items, int count, int op) {
  size_t bytes = 0;
  const auto align = [](size_t v) { return (v + 255) / 256 * 256; };
  bytes += align(sizeof(BatchControl));
  if (op == BSM_BATCH_DHAT)
    for (int k = 0; k < count; ++k) {
      const Geom g = make_geom(items[k].lat);
      bytes += align(half_spinor_bytes(g.Vh, items[k].lat.N, BSM_F32) * items[k].nrhs);
    }
  return bytes;
}

int batch_status(void* ws, cudaStream_t s);

// builds the tasks of a D or Dhat batch for the configuration and enqueues the launch
int batch_launch_cfg(const bsm_batch_item* items, int count, const bsm_batch_opts& o, void* ws, cudaStream_t s,
                     const BatchConfig& cfg) {
  const auto align = [](size_t v) { return (v + 255) / 256 * 256; };
  char* w = reinterpret_cast<char*>(ws);
  BatchControl* ctl = reinterpret_cast<BatchControl*>(w);
  w += align(sizeof(BatchControl));

  std::vector<BatchTask> tasks, tasks1;  // phase 0 and phase 1 (the kernel wants them by phase)
  BatchMeta meta;
  memset(&meta, 0, sizeof(meta));
  meta.nphases = o.op == BSM_BATCH_DHAT ? 2 : 1;
  for (int k = 0; k < count; ++k) {
    const bsm_batch_item& it = items[k];
    const OpCtx c = make_ctx(it.lat, it.U_rep, BSM_F32, s);
    const size_t half = c.half_bytes * it.nrhs;
    const char* in = reinterpret_cast<const char*>(it.in);
    char* out = reinterpret_cast<char*>(it.out);
    const long long chunks = ((long long)c.g.Vh * (it.nrhs / cfg.rb) + kHopThreads - 1) / kHopThreads;
    BatchTask t;
    memset(&t, 0, sizeof(t));
    t.d = c.d;
    t.args.g = c.g;
    t.args.nrhs = it.nrhs;
    t.args.dagger = 0;
    t.chunks = chunks;
    if (o.op == BSM_BATCH_D) {  // out_p = A in_p - 1/2 H in_{1-p}, both parities in phase 0
      for (int p = 0; p < 2; ++p) {
        t.args.links = c.links + (size_t)p * c.link_block;
        t.args.p = p;
        t.args.in = in + (size_t)(1 - p) * half;
        t.args.out = out + (size_t)p * half;
        t.args.x = in + (size_t)p * half;
        t.args.a = c.A;
        t.args.b = -0.5;
        t.phase = 0;
        t.chunk0 = meta.phase_chunks[0];
        meta.phase_chunks[0] += chunks;
        tasks.push_back(with_tasks_scalars(t));
      }
    } else {  // phase 0: tmp_o = H_oe in_e ; phase 1: out_e = A in_e - 1/(4A) H_eo tmp_o
      char* tmp = w;
      w += align(half);
      t.args.links = c.links + c.link_block;
      t.args.p = 1;
      t.args.in = in;
      t.args.out = tmp;
      t.args.x = nullptr;
      t.args.a = 0.0;
      t.args.b = 1.0;
      t.phase = 0;
      t.chunk0 = meta.phase_chunks[0];
      meta.phase_chunks[0] += chunks;
      tasks.push_back(with_tasks_scalars(t));
      t.args.links = c.links;
      t.args.p = 0;
      t.args.in = tmp;
      t.args.out = out;
      t.args.x = in;
      t.args.a = c.A;
      t.args.b = -1.0 / (4.0 * c.A);
      t.phase = 1;
      t.chunk0 = meta.phase_chunks[1];
      meta.phase_chunks[1] += chunks;
      tasks1.push_back(with_tasks_scalars(t));
    }
  }
  tasks.insert(tasks.end(), tasks1.begin(), tasks1.end());
  return launch_tasks(tasks, meta, ctl, o.timeout_s, o.barrier_extra, cfg, s);
}

// the even-odd normal operator Mp = Dhat^+ Dhat p of every item in one
// launch of four phases: t = H_oe p, u = A p - H_eo t / (4A), t = H_oe^+ u,
// Mp = A u - H_eo^+ t / (4A); FP32 multi-RHS fields (validated by the caller)
int batch_normal_launch_cfg(const BatchNormalItem* items, int count, void* ctl_ws, double timeout_s, cudaStream_t s,
                            const BatchConfig& cfg) {
  BatchMeta meta;
  memset(&meta, 0, sizeof(meta));
  meta.nphases = 4;
  std::vector<BatchTask> by_phase[4];
  for (int k = 0; k < count; ++k) {
    const BatchNormalItem& it = items[k];
    const OpCtx c = make_ctx(it.lat, it.U32, BSM_F32, s);
    BatchTask t;
    memset(&t, 0, sizeof(t));
    t.d = c.d;
    t.args.g = c.g;
    t.args.nrhs = it.nrhs;
    t.chunks = ((long long)c.g.Vh * (it.nrhs / cfg.rb) + kHopThreads - 1) / kHopThreads;
    for (int ph = 0; ph < 4; ++ph) {
      const bool first_hop = (ph & 1) == 0;  // phases 0, 2: tmp_o = H_oe(^+) v
      const void* v = ph < 2 ? it.p : it.u;
      t.args.dagger = ph >= 2;
      t.args.p = first_hop ? 1 : 0;
      t.args.links = c.links + (size_t)t.args.p * c.link_block;
      t.args.in = first_hop ? v : it.t;
      t.args.out = first_hop ? it.t : (ph == 1 ? it.u : it.Mp);
      t.args.x = first_hop ? nullptr : v;
      t.args.a = first_hop ? 0.0 : c.A;
      t.args.b = first_hop ? 1.0 : -1.0 / (4.0 * c.A);
      t.phase = ph;
      t.chunk0 = meta.phase_chunks[ph];
      meta.phase_chunks[ph] += t.chunks;
      by_phase[ph].push_back(with_tasks_scalars(t));
    }
  }
  std::vector<BatchTask> tasks;
  for (int ph = 0; ph < 4; ++ph) tasks.insert(tasks.end(), by_phase[ph].begin(), by_phase[ph].end());
  return launch_tasks(tasks, meta, reinterpret_cast<BatchControl*>(ctl_ws), timeout_s, 0, cfg, s);
}

namespace {

// --- launch-configuration tuner: per batch shape, the first call times every
// (RB, grab) candidate on the caller's stream and keeps the fastest ---------
std::mutex g_tune_mu;
std::map<std::string, BatchConfig> g_tuned;
thread_local BatchConfig g_last;

bool tuning_allowed(cudaStream_t s) {
  const char* env = getenv("BSM_BATCH_TUNE");
  if (env != nullptr && env[0] == '0') return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
  return true;
}

// candidates: RHS blocks 1 and 2, and packed pairs of 2 and 4 RHS, where
// every lattice's nrhs is a multiple of the block; with every grab size
// BSM_BATCH_CONFIG="rb:grab" (rb = 1, 2, 102 or 104) pins the configuration
// for every shape whose nrhs allow it; false if it is unset or malformed
bool pinned_config(int nrhs_gcd, BatchConfig& cfg) {
  const char* env = getenv("BSM_BATCH_CONFIG");
  int rb = 0, grab = 0;
  if (env == nullptr || sscanf(env, "%d:%d", &rb, &grab) != 2) return false;
  const bool paired = rb == kPairedBlock + 2 || rb == kPairedBlock + 4;
  if (paired) rb -= kPairedBlock;
  if (!(rb == 1 || rb == 2 || (paired && rb == 4)) || !(grab == 1 || grab == 2 || grab == 4 || grab == 8) ||
      nrhs_gcd % rb != 0)
    return false;
  cfg.rb = rb;
  cfg.grab = grab;
  cfg.paired = paired;
  return true;
}

template <typename Launch>
int tuned_launch(const std::string& key, int nrhs_gcd, cudaStream_t s, void* ctl_ws, Launch launch) {
  BatchConfig cfg;
  if (pinned_config(nrhs_gcd, cfg)) {
    g_last = cfg;
    return launch(cfg);
  }
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      cfg = it->second;
      have = true;
    }
  }
  if (!have && tuning_allowed(s)) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BSM_ECUDA;
    float best = 1e30f;
    BatchConfig win;
    const BatchConfig blocks[4] = {{1, 4, false}, {2, 4, false}, {2, 4, true}, {4, 4, true}};
    for (const BatchConfig& blk : blocks) {
      if (nrhs_gcd % blk.rb != 0) continue;
      for (int grab : {1, 2, 4, 8}) {
        BatchConfig c = blk;
        c.grab = grab;
        int rc = launch(c);  // warm-up
        float ms = 0.f, tot = 0.f;
        for (int r = 0; r < 3 && rc == BSM_OK; ++r) {
          cudaEventRecord(e0, s);
          rc = launch(c);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = BSM_ECUDA;
          tot += ms;
        }
        if (rc == BSM_OK) rc = batch_status(ctl_ws, s);
        if (rc != BSM_OK) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return rc;
        }
        if (tot < best) {
          best = tot;
          win = c;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cfg = win;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = cfg;
  }
  g_last = cfg;
  return launch(cfg);
}

std::string shape_key(const char* op, const bsm_lattice* lats, const int* nrhs, int count, size_t stride) {
  std::string k(op);
  for (int i = 0; i < count; ++i) {
    const bsm_lattice& L = *reinterpret_cast<const bsm_lattice*>(reinterpret_cast<const char*>(lats) + i * stride);
    const int n = *reinterpret_cast<const int*>(reinterpret_cast<const char*>(nrhs) + i * stride);
    char buf[96];
    snprintf(buf, sizeof(buf), "|%d,%d,%d,%d:%d:%d", L.dims[0], L.dims[1], L.dims[2], L.dims[3], L.N, n);
    k += buf;
  }
  return k;
}

}  // namespace

// launches the batch on `s`; with sync, waits and reads the error flag
// (BSM_ETIMEOUT), else returns at once (nothing but a memset and the
// cooperative launch is enqueued, so the call can be captured in a graph).
// The first call per batch shape tunes the launch configuration (which
// synchronises `s`) unless the stream is capturing or BSM_BATCH_TUNE=0.
int batch_launch(const bsm_batch_item* items, int count, const bsm_batch_opts& o, void* ws, cudaStream_t s,
                 bool sync) {
  int gcd = 0;
  for (int k = 0; k < count; ++k) gcd = std::gcd(gcd, (int)items[k].nrhs);
  const std::string key = shape_key(o.op == BSM_BATCH_DHAT ? "dhat" : "d", &items[0].lat, &items[0].nrhs, count,
                                    sizeof(bsm_batch_item));
  const int rc = tuned_launch(key, gcd, s, ws,
                              [&](const BatchConfig& c) { return batch_launch_cfg(items, count, o, ws, s, c); });
  if (rc != BSM_OK) return rc;
  return sync ? batch_status(ws, s) : BSM_OK;
}

int batch_normal_launch(const BatchNormalItem* items, int count, void* ctl_ws, double timeout_s, cudaStream_t s) {
  int gcd = 0;
  for (int k = 0; k < count; ++k) gcd = std::gcd(gcd, items[k].nrhs);
  const std::string key = shape_key("normal", &items[0].lat, &items[0].nrhs, count, sizeof(BatchNormalItem));
  return tuned_launch(key, gcd, s, ctl_ws, [&](const BatchConfig& c) {
    return batch_normal_launch_cfg(items, count, ctl_ws, timeout_s, s, c);
  });
}

// RHS per thread as the multi-RHS block codes: 1, 2, or 102, 104 for packed pairs
void batch_last_config(int* rb, int* grab) {
  *rb = g_last.paired ? kPairedBlock + g_last.rb : g_last.rb;
  *grab = g_last.grab;
}

size_t batch_control_bytes() { return (sizeof(BatchControl) + 255) / 256 * 256; }

// waits for `s` and reads the error flag the last batch on this workspace left
int batch_status(void* ws, cudaStream_t s) {
  const BatchControl* ctl = reinterpret_cast<const BatchControl*>(ws);
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return err ? BSM_ETIMEOUT : BSM_OK;
}

}  // namespace bsm
