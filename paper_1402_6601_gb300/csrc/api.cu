// Library-wide entry points: defaults, device queries, and host introspection of the task
// graph and of the activate policies (the same code the persistent kernel runs).
#include <mutex>
#include <set>
#include <tuple>
#include <vector>
#include "common.cuh"
#include "dag.cuh"
#include "dag_lu.cuh"
#include "internal.cuh"
#include "sched.cuh"

namespace chol {

DeviceInfo current_device_info() {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  DeviceInfo di;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return di;
  }
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() > dev && cache[dev].device == dev) return cache[dev];
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return di;
  }
  di.device = dev;
  di.sms = p.multiProcessorCount;
  di.cc_major = p.major;
  di.cc_minor = p.minor;
  di.smem_optin = p.sharedMemPerBlockOptin;
  if ((int)cache.size() <= dev) cache.resize(dev + 1);
  cache[dev] = di;
  return di;
}

cudaError_t set_smem_attr(const void *fn, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<const void *, int, int>> done;  // (kernel, device, bytes)
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(fn, dev, bytes);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  done.insert(key);
  return cudaSuccess;
}

// One thread of a warp-wide placement on the device, for chol_sched_activate_device.
__global__ void sched_activate_kernel(int policy, double alpha, int max_iter, double eps, int m,
                                      const int *tid, const long long *p, const long long *prio,
                                      const int *aff, const long long *score, int use_cp,
                                      const long long *comm, const int *own3, const int *nin, int W,
                                      const long long *load_in, int *out_tid, int *out_worker,
                                      int *out_iters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ReadyTask *LR = reinterpret_cast<ReadyTask *>(smem_raw);
  size_t off = align_up((size_t)m * sizeof(ReadyTask), 16);
  int *ints = reinterpret_cast<int *>(smem_raw + off);
  PlaceScratch ps;
  ps.ord_prio = ints;
  ps.ord_aff = ints + m;
  ps.ord_lpt = ints + 2 * m;
  ps.assign = ints + 3 * m;
  ps.trial = ints + 4 * m;
  off += align_up((size_t)m * 4 * 5, 16);
  int64_t *load = reinterpret_cast<int64_t *>(smem_raw + off);
  ps.tload = load + W;
  const int lane = threadIdx.x;
  for (int i = lane; i < m; i += 32) {
    LR[i].tid = tid[i];
    LR[i].p = p[i];
    LR[i].prio = prio[i];
    LR[i].aff = aff[i];
    LR[i].score = score[i];
    LR[i].comm = use_cp ? comm[i] : 0;
    LR[i].nin = use_cp ? nin[i] : 0;
    for (int a = 0; a < 3; ++a) LR[i].own[a] = use_cp ? own3[3 * i + a] : -1;
  }
  for (int w = lane; w < W; w += 32) load[w] = load_in[w];
  __syncwarp();
  const int it = place<WarpExec>(policy, alpha, max_iter, eps, LR, m, load, W, ps, use_cp != 0);
  __syncwarp();
  for (int q = lane; q < m; q += 32) {
    const int i = ps.ord_prio[q];
    out_tid[q] = LR[i].tid;
    out_worker[q] = ps.assign[i];
  }
  if (lane == 0) *out_iters = it;
}

static size_t sched_smem(int m, int W) {
  return align_up((size_t)m * sizeof(ReadyTask), 16) + align_up((size_t)m * 4 * 5, 16) +
         (size_t)W * 16;
}

}  // namespace chol

using namespace chol;

extern "C" const char *chol_version(void) { return "paper_1402_6601_gb300 0.1 (sm_103a)"; }

extern "C" void chol_opts_default(chol_opts *o) {
  if (!o) return;
  o->nb = 0;  // automatic by n
  o->policy = CHOL_POLICY_HEFT;
  o->alpha = 0.5;
  o->steal = 1;
  o->workers_per_sm = 2;
  o->num_workers = 0;
  o->queue_order = 0;
  o->dada_max_iter = 16;
  o->dada_eps = 0.01;
  for (int k = 0; k < 4; ++k) o->cost_ns[k] = 0;
  o->timeout_ns = 10000000000ll;
  o->trace = 0;
  o->hold_task = -1;
  o->use_cp = 0;
  o->cp_gbs = 40.0;
  o->split = 1;
  o->keep_next = 1;
}

extern "C" size_t chol_opts_size(void) { return sizeof(chol_opts); }

extern "C" long long chol_dag_task_count(int T) {
  if (T < 1 || T > 1024) return -1;
  return task_count(T);
}

extern "C" long long chol_dag_edge_count(int T) {
  if (T < 1 || T > 1024) return -1;
  return edge_count(T);
}

template <class G>
static chol_status describe_graph(int T, int *kind, int *ti, int *tj, int *tk, int *indeg, long long *succ_ptr,
                                  long long *succ) {
  if (T < 1 || T > 1024) return CHOL_ERR_INVALID_ARG;
  const int64_t nt = G::count(T);
  int64_t e = 0;
  for (int64_t id = 0; id < nt; ++id) {
    const TaskDesc d = G::desc(T, id);
    if (kind) kind[id] = d.kind;
    if (ti) ti[id] = d.i;
    if (tj) tj[id] = d.j;
    if (tk) tk[id] = d.k;
    if (indeg) indeg[id] = G::initial(d);
    if (succ_ptr) succ_ptr[id] = e;
    const int ns = G::nsucc(T, d);
    for (int s = 0; s < ns; ++s, ++e)
      if (succ) succ[e] = G::succ(T, d, s);
  }
  if (succ_ptr) succ_ptr[nt] = e;
  return CHOL_OK;
}

extern "C" chol_status chol_dag_describe(int T, int *kind, int *ti, int *tj, int *tk, int *indeg,
                                         long long *succ_ptr, long long *succ) {
  return describe_graph<CholGraph>(T, kind, ti, tj, tk, indeg, succ_ptr, succ);
}

extern "C" long long chol_lu_dag_task_count(int T) {
  if (T < 1 || T > 1024) return -1;
  return LuGraph::count(T);
}

extern "C" chol_status chol_lu_dag_describe(int T, int *kind, int *ti, int *tj, int *tk, int *indeg,
                                            long long *succ_ptr, long long *succ) {
  return describe_graph<LuGraph>(T, kind, ti, tj, tk, indeg, succ_ptr, succ);
}

extern "C" chol_status chol_lu_dag_bottom_levels(int T, const long long *cost_ns, long long *bl) {
  if (T < 1 || T > 1024 || !cost_ns || !bl) return CHOL_ERR_INVALID_ARG;
  const int64_t cost[4] = {cost_ns[0], cost_ns[1], cost_ns[2], cost_ns[3]};
  int64_t *b = reinterpret_cast<int64_t *>(bl);
  // every successor has a larger id: reverse id order
  for (int64_t id = LuGraph::count(T) - 1; id >= 0; --id) b[id] = LuGraph::bottom_level_of(T, LuGraph::desc(T, id), cost, b);
  return CHOL_OK;
}

extern "C" chol_status chol_dag_bottom_levels_device(int lu, int T, const long long *cost_ns, long long *dBl,
                                                     void *stream) {
  if (T < 1 || T > 1024 || !cost_ns || !dBl) return CHOL_ERR_INVALID_ARG;
  const int64_t cost[4] = {cost_ns[0], cost_ns[1], cost_ns[2], cost_ns[3]};
  return bottom_levels_device(lu != 0, T, cost, reinterpret_cast<int64_t *>(dBl), (cudaStream_t)stream);
}

extern "C" chol_status chol_dag_bottom_levels(int T, const long long *cost_ns, long long *bl) {
  if (T < 1 || T > 1024 || !cost_ns || !bl) return CHOL_ERR_INVALID_ARG;
  const int64_t cost[4] = {cost_ns[0], cost_ns[1], cost_ns[2], cost_ns[3]};
  const int64_t nt = task_count(T);
  // every successor has a larger id than its predecessor except inside a step, where the
  // order GEMM/SYRK, TRSM, POTRF is used (as on the device)
  int64_t *b = reinterpret_cast<int64_t *>(bl);
  for (int k = T - 1; k >= 0; --k) {
    const int64_t base = step_offset(T, k);
    const int64_t m = T - 1 - k;
    for (int64_t id = base + 1 + m; id < base + step_size(m); ++id)
      b[id] = bottom_level_of(T, task_desc(T, id), cost, b);
    for (int64_t id = base + 1; id <= base + m; ++id)
      b[id] = bottom_level_of(T, task_desc(T, id), cost, b);
    b[base] = bottom_level_of(T, task_desc(T, base), cost, b);
  }
  (void)nt;
  return CHOL_OK;
}

extern "C" chol_status chol_sched_activate(int policy, double alpha, int max_iter, double eps,
                                           int m, const int *tid, const long long *p,
                                           const long long *prio, const int *aff,
                                           const long long *score, int use_cp, const long long *comm,
                                           const int *own3, const int *nin, int W, const long long *load,
                                           int *out_tid, int *out_worker, int *out_iters) {
  if ((policy != CHOL_POLICY_HEFT && policy != CHOL_POLICY_DADA) || m < 0 || m > 1024 || W < 1 ||
      W > 1024 || !(alpha >= 0.0 && alpha <= 1.0) || max_iter < 0 || !(eps >= 0.0))
    return CHOL_ERR_INVALID_ARG;
  if (m > 0 && (!tid || !p || !prio || !aff || !score || !out_tid || !out_worker)) return CHOL_ERR_INVALID_ARG;
  if (m > 0 && use_cp && (!comm || !own3 || !nin)) return CHOL_ERR_INVALID_ARG;
  if (!load) return CHOL_ERR_INVALID_ARG;
  std::vector<ReadyTask> LR(m > 0 ? m : 1);
  for (int i = 0; i < m; ++i) {
    LR[i].tid = tid[i];
    LR[i].p = p[i];
    LR[i].prio = prio[i];
    LR[i].aff = aff[i];
    LR[i].score = score[i];
    LR[i].comm = use_cp ? comm[i] : 0;
    LR[i].nin = use_cp ? nin[i] : 0;
    for (int a = 0; a < 3; ++a) LR[i].own[a] = use_cp ? own3[3 * i + a] : -1;
  }
  std::vector<int> ints(5 * (m > 0 ? m : 1));
  std::vector<int64_t> ld(2 * W);
  for (int w = 0; w < W; ++w) ld[w] = load[w];
  PlaceScratch ps;
  ps.ord_prio = ints.data();
  ps.ord_aff = ints.data() + m;
  ps.ord_lpt = ints.data() + 2 * m;
  ps.assign = ints.data() + 3 * m;
  ps.trial = ints.data() + 4 * m;
  ps.tload = ld.data() + W;
  const int it = place<HostExec>(policy, alpha, max_iter, eps, LR.data(), m, ld.data(), W, ps, use_cp != 0);
  for (int q = 0; q < m; ++q) {
    const int i = ps.ord_prio[q];
    out_tid[q] = LR[i].tid;
    out_worker[q] = ps.assign[i];
  }
  if (out_iters) *out_iters = it;
  return CHOL_OK;
}

extern "C" chol_status chol_sched_activate_device(int policy, double alpha, int max_iter, double eps,
                                                  int m, const int *dtid, const long long *dp,
                                                  const long long *dprio, const int *daff,
                                                  const long long *dscore, int use_cp,
                                                  const long long *dcomm, const int *down3,
                                                  const int *dnin, int W, const long long *dload,
                                                  int *dout_tid, int *dout_worker, int *dout_iters,
                                                  void *stream) {
  if ((policy != CHOL_POLICY_HEFT && policy != CHOL_POLICY_DADA) || m < 1 || m > 1024 || W < 1 ||
      W > 1024 || !(alpha >= 0.0 && alpha <= 1.0) || max_iter < 0 || !(eps >= 0.0))
    return CHOL_ERR_INVALID_ARG;
  if (!dtid || !dp || !dprio || !daff || !dscore || !dload || !dout_tid || !dout_worker || !dout_iters)
    return CHOL_ERR_INVALID_ARG;
  if (use_cp && (!dcomm || !down3 || !dnin)) return CHOL_ERR_INVALID_ARG;
  const size_t smem = sched_smem(m, W);
  CHOL_CUDA_TRY(cudaFuncSetAttribute(sched_activate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  sched_activate_kernel<<<1, 32, smem, (cudaStream_t)stream>>>(policy, alpha, max_iter, eps, m, dtid, dp,
                                                                dprio, daff, dscore, use_cp, dcomm, down3,
                                                                dnin, W, dload, dout_tid, dout_worker,
                                                                dout_iters);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

// ------------------------------------------------------------------------------------
// Host-buffer factor + solve (LAPACK dposv semantics) through a caller-provided stage.

namespace {
struct StageLayout {
  size_t a, b, fwork, swork, info, total, fbytes, sbytes;
};
StageLayout stage_layout(int n, int nrhs, const chol_opts *opts) {
  StageLayout s;
  size_t o = 0;
  s.a = o; o += chol::align_up((size_t)n * n * 8, 256);
  s.b = o; o += chol::align_up((size_t)n * nrhs * 8, 256);
  s.fbytes = chol_factor_workspace_size(n, opts);
  s.fwork = o; o += chol::align_up(s.fbytes, 256);
  s.sbytes = chol_solve_workspace_size(n, nrhs);
  s.swork = o; o += chol::align_up(s.sbytes, 256);
  s.info = o; o += 256;
  s.total = o;
  return s;
}
}  // namespace

extern "C" size_t chol_posv_host_stage_size(int n, int nrhs, const chol_opts *opts) {
  if (n < 0 || nrhs < 0) return 0;
  return stage_layout(n, nrhs, opts).total;
}

extern "C" chol_status chol_posv_host(int n, int nrhs, double *hA, int lda, double *hB, int ldb,
                                      const chol_opts *opts, void *dStage, size_t stage_bytes,
                                      int *hInfo, void *stream) {
  if (n < 0 || nrhs < 0 || !hInfo || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1))
    return CHOL_ERR_INVALID_ARG;
  if (n > 0 && (!hA || (nrhs > 0 && !hB))) return CHOL_ERR_INVALID_ARG;
  *hInfo = 0;
  if (n == 0) return CHOL_OK;
  const StageLayout L = stage_layout(n, nrhs, opts);
  if (L.fbytes == 0) return CHOL_ERR_INVALID_ARG;
  if (!dStage || stage_bytes < L.total || ((uintptr_t)dStage & 255)) return CHOL_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *st = static_cast<unsigned char *>(dStage);
  double *dA = reinterpret_cast<double *>(st + L.a);
  double *dB = reinterpret_cast<double *>(st + L.b);
  int *dInfo = reinterpret_cast<int *>(st + L.info);
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(dA, (size_t)n * 8, hA, (size_t)lda * 8, (size_t)n * 8, n,
                                  cudaMemcpyHostToDevice, s));
  if (nrhs > 0)
    CHOL_CUDA_TRY(cudaMemcpy2DAsync(dB, (size_t)n * 8, hB, (size_t)ldb * 8, (size_t)n * 8, nrhs,
                                    cudaMemcpyHostToDevice, s));
  chol_status r = chol_factor(n, dA, n, opts, st + L.fwork, L.fbytes, dInfo, stream);
  if (r != CHOL_OK) return r;
  CHOL_CUDA_TRY(cudaMemcpyAsync(hInfo, dInfo, sizeof(int), cudaMemcpyDeviceToHost, s));
  CHOL_CUDA_TRY(cudaStreamSynchronize(s));
  const int info = *hInfo;
  if (info == 0 && nrhs > 0) {
    r = chol_solve(n, nrhs, dA, n, dB, n, st + L.swork, L.sbytes, dInfo, stream);
    if (r != CHOL_OK) return r;
    CHOL_CUDA_TRY(cudaMemcpy2DAsync(hB, (size_t)ldb * 8, dB, (size_t)n * 8, (size_t)n * 8, nrhs,
                                    cudaMemcpyDeviceToHost, s));
    CHOL_CUDA_TRY(cudaMemcpyAsync(hInfo, dInfo, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  CHOL_CUDA_TRY(cudaMemcpy2DAsync(hA, (size_t)lda * 8, dA, (size_t)n * 8, (size_t)n * 8, n,
                                  cudaMemcpyDeviceToHost, s));
  CHOL_CUDA_TRY(cudaStreamSynchronize(s));
  if (*hInfo > 0) return CHOL_ERR_NOT_SPD;
  if (*hInfo < 0) return CHOL_ERR_TIMEOUT;
  return CHOL_OK;
}
