// gr_batch.cu — many BFS / SSSP jobs over many graphs in one persistent launch.
//
// Batching the paper's primitives: instead of one cooperative grid per query
// (whose per-level barrier costs dominate small graphs), a single persistent
// launch holds one job per thread-block cluster.  A cluster takes the next
// job from a device counter (jobs sorted largest first, so the longest jobs
// start earliest), runs the same BFS / SSSP body as the single-query kernels
// with the cluster as its thread scope — the step barrier is the hardware
// cluster barrier, co-scheduling of a cluster's CTAs is guaranteed by the
// hardware — and then takes the next job.  Every cluster owns one scratch
// slot (queues, chunk lists, bitmaps, keys, counters) sized for the largest
// graph of the batch.  The launch (with the resets of the job counter and of
// the per-job status words) can be captured once into a CUDA graph and
// replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gr_bfs_body.cuh"
#include "gr_sssp_body.cuh"

namespace {

struct DevJob {
  const int32_t* R;
  const int32_t* C;
  const uint32_t* W;
  int64_t m;
  int32_t n;
  int32_t op;
  int32_t src;
  int32_t flags;
  int32_t max_degree;
  int32_t big;
  int32_t* out;
  int32_t* pred;
  float do_a, do_b;
  uint32_t delta;
  int32_t index;  // position in the caller's job array (status slot)
};

struct BatchArgs {
  const DevJob* jobs;
  int njobs;
  int* next_job;
  unsigned char* scratch;
  size_t slot_bytes;
  int32_t nmax;
  int64_t chunk_cap;
  int* job_status;
  unsigned spin;
};

// slot layout (byte offsets, 256-aligned)
struct SlotLayout {
  size_t ctl, job, q0, q1, qm0, qm1, ul0, ul1, ch0, ch1, vis, fr0, fr1, fr2, key, far0, far1,
      stn, stf, total;
};

size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

SlotLayout slot_layout(int32_t nmax, int64_t chunk_cap) {
  SlotLayout L;
  const size_t nq = r256(((size_t)nmax + 1) * 4);
  const size_t nc = r256((size_t)chunk_cap * 8);
  const size_t nb = r256((((size_t)nmax + 31) / 32 + 1) * 4);
  const size_t nk = r256(((size_t)nmax + 1) * 8);
  size_t o = 0;
  L.ctl = o; o += r256(sizeof(GrCtl));
  L.job = o; o += 256;
  L.q0 = o; o += nq;
  L.q1 = o; o += nq;
  L.qm0 = o; o += nq;
  L.qm1 = o; o += nq;
  L.ul0 = o; o += nq;
  L.ul1 = o; o += nq;
  L.ch0 = o; o += nc;
  L.ch1 = o; o += nc;
  L.vis = o; o += nb;
  L.fr0 = o; o += nb;
  L.fr1 = o; o += nb;
  L.fr2 = o; o += nb;
  L.key = o; o += nk;
  L.far0 = o; o += nq;
  L.far1 = o; o += nq;
  L.stn = o; o += nq;
  L.stf = o; o += nq;
  L.total = o;
  return L;
}

__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

constexpr int BT = 256;

__global__ void __launch_bounds__(BT) batch_kernel(BatchArgs b, SlotLayout L) {
  const unsigned csize = cluster_nctarank();
  const unsigned crank = cluster_ctarank();
  const unsigned slot = blockIdx.x / csize;
  __shared__ GrArena ar;  // staging buffers, shared by the BFS and SSSP bodies
  unsigned char* base = b.scratch + (size_t)slot * b.slot_bytes;
  GrCtl* ctl = (GrCtl*)(base + L.ctl);
  int* job_cell = (int*)(base + L.job);
  for (;;) {
    // rank 0 takes the next job and clears the slot's control block
    if (crank == 0) {
      int* c = (int*)ctl;
      for (int i = threadIdx.x; i < (int)(sizeof(GrCtl) / sizeof(int)); i += BT) c[i] = 0;
      if (threadIdx.x == 0) *job_cell = atomicAdd(b.next_job, 1);
    }
    cluster_barrier();
    const int j = __ldcg(job_cell);
    if (j >= b.njobs) break;
    const DevJob& J = b.jobs[j];
    ClusterScope sc{ctl, (int64_t)crank * BT + threadIdx.x, (int64_t)csize * BT};
    if (J.op == GR_OP_BFS) {
      BfsArgs a = {};
      a.n = J.n;
      a.m = J.m;
      a.R = J.R;
      a.C = J.C;
      a.depth = J.out;
      a.pred = J.pred;
      a.visited = (uint32_t*)(base + L.vis);
      a.front[0] = (uint32_t*)(base + L.fr0);
      a.front[1] = (uint32_t*)(base + L.fr1);
      a.front[2] = (uint32_t*)(base + L.fr2);
      a.q[0] = (int32_t*)(base + L.q0);
      a.q[1] = (int32_t*)(base + L.q1);
      a.qm[0] = (int32_t*)(base + L.qm0);
      a.qm[1] = (int32_t*)(base + L.qm1);
      a.ulist[0] = (int32_t*)(base + L.ul0);
      a.ulist[1] = (int32_t*)(base + L.ul1);
      a.ch[0] = (int2*)(base + L.ch0);
      a.ch[1] = (int2*)(base + L.ch1);
      a.chunk_cap = b.chunk_cap;
      a.ctl = ctl;
      a.status = &b.job_status[J.index];
      a.src = J.src;
      a.nwords = (int32_t)(((int64_t)J.n + 31) / 32);
      a.use_do = (J.flags & GR_SYMMETRIC) ? 1 : 0;
      a.force_pull = 0;
      a.big = J.big;
      a.track_deg = a.use_do || J.max_degree >= GR_MEDIUM_DEGREE;
      a.do_a = J.do_a;
      a.do_b = J.do_b;
      a.spin = b.spin;
      a.bulk_edges = 0;  // batched graphs are small: every push level claims as it goes
      gr_bfs_body<true>(a, sc, ar);
    } else {
      SsspArgs a = {};
      a.n = J.n;
      a.R = J.R;
      a.C = J.C;
      a.W = J.W;
      a.key = (unsigned long long*)(base + L.key);
      a.dist = (uint32_t*)J.out;
      a.pred = J.pred;
      a.q[0] = (int32_t*)(base + L.q0);
      a.q[1] = (int32_t*)(base + L.q1);
      a.qm[0] = (int32_t*)(base + L.qm0);
      a.qm[1] = (int32_t*)(base + L.qm1);
      a.ch[0] = (int2*)(base + L.ch0);
      a.ch[1] = (int2*)(base + L.ch1);
      a.chunk_cap = b.chunk_cap;
      a.far[0] = (int32_t*)(base + L.far0);
      a.far[1] = (int32_t*)(base + L.far1);
      a.stamp_near = (int32_t*)(base + L.stn);
      a.stamp_far = (int32_t*)(base + L.stf);
      a.touched = (uint32_t*)(base + L.vis);
      a.bulk_rows = gr_default_bulk_rows(J.n);
      a.ctl = ctl;
      a.status = &b.job_status[J.index];
      a.src = J.src;
      a.delta = J.delta;
      a.big = J.big;
      a.track_deg = J.max_degree >= GR_MEDIUM_DEGREE;
      a.spin = b.spin;
      gr_sssp_body<false>(a, sc, ar);
    }
    cluster_barrier();  // the job is complete before rank 0 reuses the slot
  }
}

}  // namespace

struct gr_batch {
  int device;
  int njobs;
  DevJob* d_jobs;
  int* d_next;
  int* d_status;
  int* h_status;
  unsigned char* scratch;
  size_t slot_bytes;
  SlotLayout layout;
  BatchArgs args;
  int grid;
  int cluster;
  int use_graph;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

static uint32_t job_delta(const gr_graph* g) { return gr_default_delta(g); }

static cudaError_t batch_enqueue(gr_batch* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int) * b->njobs, s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(BT);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = b->cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_kernel, b->args, b->layout);
}

static void batch_free(gr_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* ptrs[] = {b->d_jobs, b->d_next, b->d_status, b->scratch};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b;
}

extern "C" void gr_batch_opts_default(gr_batch_opts* o) {
  if (!o) return;
  o->cluster_size = 8;
  o->clusters_per_sm = 0;
  o->use_graph = 1;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
}

extern "C" gr_status gr_batch_create(const gr_job* jobs, int32_t njobs, const gr_batch_opts* opts,
                                     gr_batch** out) {
  if (!jobs || njobs <= 0 || !out) return GR_ERR_INVALID_ARG;
  gr_batch_opts o;
  gr_batch_opts_default(&o);
  if (opts) o = *opts;
  if (o.cluster_size < 1 || o.cluster_size > 16 || o.clusters_per_sm < 0) return GR_ERR_INVALID_ARG;
  *out = nullptr;
  // validate jobs and size the scratch slots for the largest graph
  int32_t nmax = 1;
  int64_t chunk_cap = 2;
  std::vector<DevJob> hj(njobs);
  std::vector<double> cost(njobs);
  int device = -1;
  for (int i = 0; i < njobs; ++i) {
    const gr_job& J = jobs[i];
    const gr_graph* g = J.g;
    if (!g || !J.out || (J.op != GR_OP_BFS && J.op != GR_OP_SSSP) || J.src < 0 || J.src >= g->n)
      return GR_ERR_INVALID_ARG;
    if (J.op == GR_OP_SSSP && !g->W && g->m > 0) return GR_ERR_UNSUPPORTED;
    if (device < 0) device = g->device;
    if (g->device != device) return GR_ERR_INVALID_ARG;
    const int big = J.big_degree > 0 ? std::max(J.big_degree, 32)
                                     : (J.op == GR_OP_BFS ? GR_DEFAULT_BFS_BIG : GR_DEFAULT_SSSP_BIG);
    nmax = std::max(nmax, g->n);
    chunk_cap = std::max<int64_t>(chunk_cap, g->m / GR_CHUNK_EDGES + g->m / big + 2);
    DevJob d = {};
    d.R = g->R;
    d.C = g->C;
    d.W = g->W;
    d.m = g->m;
    d.n = g->n;
    d.op = J.op;
    d.src = J.src;
    d.flags = (int32_t)g->flags;
    d.max_degree = g->max_degree;
    d.big = big;
    d.out = (int32_t*)J.out;
    d.pred = J.pred;
    d.do_a = J.do_a > 0.f ? J.do_a : 0.05f;
    d.do_b = J.do_b > 0.f ? J.do_b : 0.05f;
    d.delta = J.delta ? J.delta : job_delta(g);
    d.index = i;
    hj[i] = d;
    cost[i] = (double)g->m * (J.op == GR_OP_SSSP ? 4.0 : 1.0) + (double)g->n;
  }
  // largest jobs first
  std::vector<int> order(njobs);
  for (int i = 0; i < njobs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<DevJob> sorted(njobs);
  for (int i = 0; i < njobs; ++i) sorted[i] = hj[order[i]];

  gr_batch* b = new (std::nothrow) gr_batch();
  if (!b) return GR_ERR_OOM;
  b->device = device;
  b->njobs = njobs;
  b->cluster = o.cluster_size;
  b->use_graph = o.use_graph;
  b->layout = slot_layout(nmax, chunk_cap);
  b->slot_bytes = b->layout.total;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  // resident clusters: the occupancy calculator with this cluster shape
  if (b->cluster > 8 &&
      cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    batch_free(b);
    return GR_ERR_UNSUPPORTED;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sms * 32);
  cfg.blockDim = dim3(BT);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = b->cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, batch_kernel, &cfg) != cudaSuccess ||
      clusters < 1) {
    (void)cudaGetLastError();
    batch_free(b);
    return GR_ERR_UNSUPPORTED;
  }
  if (o.clusters_per_sm > 0) {
    const int want = std::max(1, o.clusters_per_sm * sms / b->cluster);
    clusters = std::min(clusters, want);
  }
  clusters = std::min(clusters, njobs);
  b->grid = clusters * b->cluster;
  const size_t scratch = b->slot_bytes * (size_t)clusters;
  if (cudaMalloc(&b->d_jobs, sizeof(DevJob) * njobs) != cudaSuccess ||
      cudaMalloc(&b->d_next, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_status, sizeof(int) * njobs) != cudaSuccess ||
      cudaMalloc(&b->scratch, scratch) != cudaSuccess ||
      cudaMallocHost(&b->h_status, sizeof(int) * njobs) != cudaSuccess) {
    (void)cudaGetLastError();
    batch_free(b);
    return GR_ERR_OOM;
  }
  if (cudaMemcpy(b->d_jobs, sorted.data(), sizeof(DevJob) * njobs, cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    batch_free(b);
    return GR_ERR_CUDA;
  }
  b->args.jobs = b->d_jobs;
  b->args.njobs = njobs;
  b->args.next_job = b->d_next;
  b->args.scratch = b->scratch;
  b->args.slot_bytes = b->slot_bytes;
  b->args.nmax = nmax;
  b->args.chunk_cap = chunk_cap;
  b->args.job_status = b->d_status;
  b->args.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;
  if (b->use_graph) {
    cudaStream_t cs;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
      ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      cudaError_t e = ok ? batch_enqueue(b, cs) : cudaErrorUnknown;
      cudaGraph_t gph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cs, &gph);
      ok = ok && e == cudaSuccess && e2 == cudaSuccess && gph;
      if (ok) {
        b->graph = gph;
        ok = cudaGraphInstantiate(&b->exec, gph, 0) == cudaSuccess;
      } else if (gph) {
        cudaGraphDestroy(gph);
      }
      cudaStreamDestroy(cs);
    }
    if (!ok) {
      (void)cudaGetLastError();
      batch_free(b);
      return GR_ERR_CUDA;
    }
  }
  *out = b;
  return GR_OK;
}

extern "C" gr_status gr_batch_run(gr_batch* b, void* stream) {
  if (!b) return GR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = b->use_graph ? cudaGraphLaunch(b->exec, s) : batch_enqueue(b, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}

extern "C" gr_status gr_batch_status(gr_batch* b, int32_t* job_status, void* stream) {
  if (!b) return GR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * b->njobs, cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  gr_status first = GR_OK;
  for (int i = 0; i < b->njobs; ++i) {
    if (job_status) job_status[i] = b->h_status[i];
    if (first == GR_OK && b->h_status[i] != 0) first = b->h_status[i];
  }
  return first;
}

extern "C" gr_status gr_batch_info(const gr_batch* b, int32_t* clusters, int32_t* cluster_size,
                                   size_t* scratch_bytes) {
  if (!b) return GR_ERR_INVALID_ARG;
  if (clusters) *clusters = b->grid / b->cluster;
  if (cluster_size) *cluster_size = b->cluster;
  if (scratch_bytes) *scratch_bytes = b->slot_bytes * (size_t)(b->grid / b->cluster);
  return GR_OK;
}

extern "C" gr_status gr_batch_destroy(gr_batch* b) {
  if (!b) return GR_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  batch_free(b);
  return GR_OK;
}
