// Batched solves of many independent Lyapunov equations (an addition to the paper, which treats
// one equation at a time; each instance follows Alg. 1-3 and the two-pass factor of Sec. 3.3).
//
// Every instance keeps its own operator copy, ring blocks, coefficient log and history in the
// batch workspace (a lyap_handle in "external" mode); the O(nmax^2) check slots and the factor
// scratch come from a few pools shared by all instances, one per stream.  One block Lanczos
// iteration of all instances is four persistent launches per block-size group (launch_batch_step
// over a list of row tiles), captured once in a CUDA graph and replayed; the checks of the
// instances run on the pool streams, round by round, like lyap_solve's speculative batches.
#include "common.cuh"

#include <limits.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

namespace {

#ifndef LYAP_BATCH_POOLS
#define LYAP_BATCH_POOLS 12
#endif
constexpr int kPools = LYAP_BATCH_POOLS;  // most pools (streams with check and factor scratch)
constexpr int kRowChoices[3] = {1024, 4096, 16384};
// check slots of one pool: room for several checks of a large instance in one launch (their
// eigenpair iterations run side by side instead of one launch after another)
#ifndef LYAP_POOL_CHECK_GB
#define LYAP_POOL_CHECK_GB 6
#endif
constexpr size_t kPoolCheckMin = (size_t)LYAP_POOL_CHECK_GB << 30;

struct Group {
  int s = 1;
  std::vector<int> inst;
  int rows = 4096;
  int per_sm = 0;   // 0: full occupancy
  int ntiles = 0;
  size_t tile_off = 0;  // first tile of the group in the tile array
  size_t tile_cap = 0;
};

struct BatchPlan {
  std::vector<size_t> inst_off, inst_bytes;
  size_t pool_off = 0, pool_check = 0, pool_factor = 0;
  int npools = 1;
  size_t inst_arr = 0, step_arr = 0, tile_arr = 0, tile_cap = 0;
  size_t total = 0;
};

int plan_batch(int count, const lyap_csr* A, const int* s, const lyap_options& o, BatchPlan& bp) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off += lyap_align256((int64_t)bytes);
    return r;
  };
  bp.inst_off.resize(count);
  bp.inst_bytes.resize(count);
  size_t slot_full = 0, fac = 0;
  // the batched sweeps run the fp64 and fp32 bulk types
  if (o.precision != LYAP_PREC_F64 && o.precision != LYAP_PREC_MIXED) return LYAP_ERR_ARG;
  for (int b = 0; b < count; ++b) {
    if (!valid_block(s[b])) return LYAP_ERR_ARG;
    int rc = validate_csr(&A[b]);
    if (rc != LYAP_OK) return rc;
    Plan p;
    rc = make_plan(&A[b], nullptr, s[b], o, p, 1);
    if (rc != LYAP_OK) return rc;
    bp.inst_bytes[b] = p.total;
    bp.inst_off[b] = take(p.total);
    const int nmax = s[b] * o.maxit;
    slot_full = std::max(slot_full, check_slot_bytes(s[b], nmax));
    fac = std::max(fac, factor_ws_bytes(s[b], nmax, 0) +
                            pass2_ws_bytes(A[b].n, s[b], o.pass2_blocks, o.precision));
    bp.tile_cap += (size_t)((A[b].n + kRowChoices[0] - 1) / kRowChoices[0]) + 1;
  }
  bp.pool_check = lyap_align256((int64_t)std::max(slot_full, kPoolCheckMin));
  bp.pool_factor = lyap_align256((int64_t)fac);
  bp.npools = std::min(kPools, count);
  bp.pool_off = take(bp.npools * (bp.pool_check + bp.pool_factor));
  bp.inst_arr = take(sizeof(BInst) * (size_t)count);
  bp.step_arr = take(sizeof(int) * 2 * (size_t)count);
  bp.tile_arr = take(sizeof(BTile) * bp.tile_cap);
  bp.total = off;
  return LYAP_OK;
}

}  // namespace

struct lyap_batch {
  int count = 0;
  lyap_options opt;
  BatchPlan plan;
  char* ws = nullptr;
  std::vector<lyap_handle*> h;
  std::vector<int> s, status, m, done;
  std::vector<Group> groups;
  std::vector<BInst> inst;
  std::vector<BTile> tiles;
  BInst* d_inst = nullptr;
  int* d_step = nullptr;
  int* h_step = nullptr;  // pinned
  BTile* d_tiles = nullptr;
  char* pool[kPools] = {};
  cudaStream_t main = nullptr;
  cudaStream_t streams[kPools] = {};
  cudaEvent_t ev[4] = {};
  cudaEvent_t join[kPools] = {};
  cudaGraphExec_t graph = nullptr;
  int sms = 0;
  int solved = 0;
  double times[8] = {};
  int64_t launches = 0;
  int64_t replays = 0;
};

namespace {

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// row tiles of group g at its configuration; per-instance tile counts go to b->inst
void build_tiles(lyap_batch* b, Group& g) {
  g.ntiles = 0;
  BTile* out = b->tiles.data() + g.tile_off;
  for (int i : g.inst) {
    const int64_t n = b->inst[i].op.n;
    int64_t rows = g.rows;
    // at most kMaxSweepGrid tiles per instance (its partials slots), multiples of the slice height
    const int64_t need = (n + kMaxSweepGrid - 1) / kMaxSweepGrid;
    if (rows < need) rows = (need + LYAP_SLICE - 1) / LYAP_SLICE * LYAP_SLICE;
    const int nt = (int)((n + rows - 1) / rows);
    for (int t = 0; t < nt; ++t) {
      BTile& tl = out[g.ntiles++];
      tl.inst = i;
      tl.local = t;
      tl.lo = (int64_t)t * rows;
      tl.hi = std::min<int64_t>(n, (int64_t)(t + 1) * rows);
    }
    b->inst[i].ntiles = nt;
  }
}

int grid_of(lyap_batch* b, const Group& g) {
  const int occ = batch_blocks_per_sm(g.s, b->opt.precision == LYAP_PREC_MIXED);
  const int per = g.per_sm > 0 ? std::min(g.per_sm, occ) : occ;
  return std::max(1, std::min(b->sms * per, std::max(1, g.ntiles)));
}

int upload(lyap_batch* b, cudaStream_t st) {
  LYAP_CUDA_TRY(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BInst) * b->count, cudaMemcpyHostToDevice, st));
  LYAP_CUDA_TRY(cudaMemcpyAsync(b->d_tiles, b->tiles.data(), sizeof(BTile) * b->plan.tile_cap, cudaMemcpyHostToDevice, st));
  return LYAP_OK;
}

int reset_steps(lyap_batch* b, cudaStream_t st) {
  for (int i = 0; i < b->count; ++i) {
    b->h_step[2 * i] = 1;
    b->h_step[2 * i + 1] = 1;
  }
  LYAP_CUDA_TRY(cudaMemcpyAsync(b->d_step, b->h_step, sizeof(int) * 2 * b->count, cudaMemcpyHostToDevice, st));
  return LYAP_OK;
}

int launch_group(lyap_batch* b, const Group& g, cudaStream_t st) {
  return launch_batch_step(g.s, b->opt.precision == LYAP_PREC_MIXED, b->d_inst, b->d_tiles + g.tile_off, g.ntiles,
                           grid_of(b, g), st);
}

// times iteration 1 of each group over the candidate tile heights and CTAs per SM
int autotune(lyap_batch* b) {
  cudaStream_t st = b->main;
  for (Group& g : b->groups) {
    const int occ = batch_blocks_per_sm(g.s, b->opt.precision == LYAP_PREC_MIXED);
    float best = 1e30f;
    int br = g.rows, bs = g.per_sm;
    for (int rows : kRowChoices)
      for (int per : {1, occ}) {
        g.rows = rows;
        g.per_sm = per;
        build_tiles(b, g);
        int rc = upload(b, st);
        if (rc != LYAP_OK) return rc;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
          if ((rc = reset_steps(b, st)) != LYAP_OK) return rc;
          cudaEventRecord(b->ev[2], st);
          b->launches += launch_group(b, g, st);
          cudaEventRecord(b->ev[3], st);
          LYAP_CUDA_TRY(cudaStreamSynchronize(st));
          LYAP_CUDA_TRY(cudaGetLastError());
          cudaEventElapsedTime(&ms, b->ev[2], b->ev[3]);
        }
        if (ms < best) {
          best = ms;
          br = rows;
          bs = per;
        }
        if (per == occ) break;  // occ == 1
      }
    g.rows = br;
    g.per_sm = bs;
  }
  return LYAP_OK;
}

int capture_graph(lyap_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t graph = nullptr;
  LYAP_CUDA_TRY(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
  for (const Group& g : b->groups) launch_group(b, g, b->main);
  LYAP_CUDA_TRY(cudaStreamEndCapture(b->main, &graph));
  const cudaError_t e = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

}  // namespace

extern "C" {

int lyap_batch_workspace_size(int count, const lyap_csr* A, const int* s, const lyap_options* opt, size_t* bytes) {
  if (count < 1 || !A || !s || !bytes) return LYAP_ERR_ARG;
  lyap_options o = resolve_options(opt);
  if (o.sell_sigma != 1) return LYAP_ERR_ARG;
  BatchPlan bp;
  int rc = plan_batch(count, A, s, o, bp);
  if (rc != LYAP_OK) return rc;
  *bytes = bp.total;
  return LYAP_OK;
}

int lyap_batch_destroy(lyap_batch* b) {
  if (!b) return LYAP_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (lyap_handle* h : b->h)
    if (h) lyap_destroy(h);
  for (int p = 0; p < kPools; ++p) {
    if (b->streams[p]) cudaStreamDestroy(b->streams[p]);
    if (b->join[p]) cudaEventDestroy(b->join[p]);
  }
  for (int i = 0; i < 4; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  if (b->main) cudaStreamDestroy(b->main);
  if (b->h_step) cudaFreeHost(b->h_step);
  delete b;
  return LYAP_OK;
}

int lyap_batch_create(int count, const lyap_csr* A, const double* const* C, int c_mem, const int* s,
                      const double* tol, const lyap_options* opt, void* workspace, size_t ws_bytes, void* stream,
                      lyap_batch** out) {
  if (!out || count < 1 || !A || !C || !s || !tol) return LYAP_ERR_ARG;
  *out = nullptr;
  lyap_options o = resolve_options(opt);
  if (o.sell_sigma != 1) return LYAP_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!C[i] || !(tol[i] >= 0.0)) return LYAP_ERR_ARG;
  BatchPlan bp;
  int rc = plan_batch(count, A, s, o, bp);
  if (rc != LYAP_OK) return rc;
  if (!workspace || ws_bytes < bp.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LYAP_ERR_WORKSPACE;
  lyap_batch* b = new (std::nothrow) lyap_batch();
  if (!b) return LYAP_ERR_ARG;
  auto fail = [&](int code) {
    lyap_batch_destroy(b);
    return code;
  };
  b->count = count;
  b->opt = o;
  b->plan = bp;
  b->ws = static_cast<char*>(workspace);
  b->sms = sm_count();
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  for (int p = 0; p < bp.npools; ++p) {
    if (cudaStreamCreateWithFlags(&b->streams[p], cudaStreamNonBlocking) != cudaSuccess) return fail(LYAP_ERR_CUDA);
    if (cudaEventCreateWithFlags(&b->join[p], cudaEventDisableTiming) != cudaSuccess) return fail(LYAP_ERR_CUDA);
    b->pool[p] = b->ws + bp.pool_off + (size_t)p * (bp.pool_check + bp.pool_factor);
  }
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&b->ev[i]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&b->h_step, sizeof(int) * 2 * count) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  cudaEventRecord(b->ev[0], user);
  cudaStreamWaitEvent(b->main, b->ev[0], 0);
  b->d_inst = reinterpret_cast<BInst*>(b->ws + bp.inst_arr);
  b->d_step = reinterpret_cast<int*>(b->ws + bp.step_arr);
  b->d_tiles = reinterpret_cast<BTile*>(b->ws + bp.tile_arr);
  b->h.assign(count, nullptr);
  b->s.assign(s, s + count);
  b->status.assign(count, LYAP_NOT_CONVERGED);
  b->m.assign(count, 0);
  b->done.assign(count, 0);
  b->inst.resize(count);
  b->tiles.resize(bp.tile_cap);
  for (int i = 0; i < count; ++i) {
    rc = create_handle(&A[i], nullptr, C[i], nullptr, c_mem, s[i], tol[i], &o, b->ws + bp.inst_off[i], bp.inst_bytes[i],
                       b->main, 1, &b->h[i]);
    if (rc != LYAP_OK) return fail(rc);
    b->h[i]->check_ws = b->pool[0];
    b->h[i]->factor_ws = b->pool[0] + bp.pool_check;
    BInst& in = b->inst[i];
    in.op = b->h[i]->op[0];
    in.flags = b->h[i]->flags;
    in.step = b->d_step + 2 * i;
    in.ntiles = 0;
    in.maxit = o.maxit;
  }
  // groups by block size; tiles at the default configuration
  size_t toff = 0;
  for (int sv : {1, 2, 3, 4, 8}) {
    Group g;
    g.s = sv;
    for (int i = 0; i < count; ++i)
      if (s[i] == sv) g.inst.push_back(i);
    if (g.inst.empty()) continue;
    g.tile_off = toff;
    for (int i : g.inst) g.tile_cap += (size_t)((A[i].n + kRowChoices[0] - 1) / kRowChoices[0]) + 1;
    toff += g.tile_cap;
    b->groups.push_back(g);
  }
  for (Group& g : b->groups) build_tiles(b, g);
  if ((rc = upload(b, b->main)) != LYAP_OK) return fail(rc);
  cudaEventRecord(b->ev[1], b->main);
  if (cudaStreamSynchronize(b->main) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
  b->times[0] = ms;
  *out = b;
  return LYAP_OK;
}

int lyap_batch_solve(lyap_batch* b, int autotune_flag, void* stream) {
  if (!b) return LYAP_ERR_ARG;
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaStream_t st = b->main;
  const lyap_options& o = b->opt;
  const int K = b->count;
  cudaEventRecord(b->ev[0], user);
  cudaStreamWaitEvent(st, b->ev[0], 0);
  cudaEventRecord(b->ev[0], st);
  for (int i = 0; i < K; ++i) {
    solve_begin(b->h[i], st);
    b->h[i]->solved = 0;
  }
  int rc = reset_steps(b, st);
  if (rc != LYAP_OK) return rc;
  if (autotune_flag) {
    if ((rc = autotune(b)) != LYAP_OK) return rc;
    for (Group& g : b->groups) build_tiles(b, g);
    if ((rc = upload(b, st)) != LYAP_OK) return rc;
    if ((rc = reset_steps(b, st)) != LYAP_OK) return rc;
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  if (!b->graph && (rc = capture_graph(b)) != LYAP_OK) return rc;
  std::vector<int> checked(K, 0), finished(K, 0);
  std::vector<std::vector<unsigned char>> was(K, std::vector<unsigned char>((size_t)o.maxit + 1, 0));
  std::vector<int> todo;
  // the checks at the m of a list for instance i, in batches that fit its pool's check area
  auto check_list = [&](int i, const std::vector<int>& ms, cudaStream_t sp) {
    lyap_handle* h = b->h[i];
    const int si = b->s[i];
    size_t a = 0;
    while (a < ms.size()) {
      size_t n = std::min(ms.size() - a, (size_t)o.check_batch);
      while (n > 1 && check_slot_bytes(si, batch_nmax(si, ms[a + n - 1])) * n > b->plan.pool_check) --n;
      h->launches += launch_check_list(h, ms.data() + a, (int)n, sp);
      for (size_t k = a; k < a + n; ++k) was[i][ms[k]] = 1;
      a += n;
    }
  };
  for (int i = 0; i < K; ++i) b->status[i] = LYAP_NOT_CONVERGED;
  int chunk = std::min(4, o.check_batch);
  float t_lanczos = 0.f, t_check = 0.f;
  int nfinished = 0;
  int64_t replays = 0;
  while (nfinished < K) {
    cudaEventRecord(b->ev[2], st);
    for (int r = 0; r < chunk; ++r) LYAP_CUDA_TRY(cudaGraphLaunch(b->graph, st));
    replays += chunk;
    cudaEventRecord(b->ev[3], st);
    LYAP_CUDA_TRY(cudaMemcpyAsync(b->h_step, b->d_step, sizeof(int) * 2 * K, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    LYAP_CUDA_TRY(cudaGetLastError());
    float a = 0.f;
    cudaEventElapsedTime(&a, b->ev[2], b->ev[3]);
    t_lanczos += a;
    // checks of the new iterations, instance by instance on the pool streams
    cudaEventRecord(b->ev[2], st);
    for (int p = 0; p < b->plan.npools; ++p) cudaStreamWaitEvent(b->streams[p], b->ev[2], 0);
    int next = 0;
    std::vector<int> pending;
    for (int i = 0; i < K; ++i) {
      if (finished[i]) continue;
      lyap_handle* h = b->h[i];
      b->done[i] = std::min(b->h_step[2 * i] - 1, o.maxit);
      if (checked[i] >= b->done[i]) continue;
      const int p = next++ % b->plan.npools;
      cudaStream_t sp = b->streams[p];
      h->check_ws = b->pool[p];
      // the history up to checked[i] is on the host (copied after the previous round)
      pick_checks(h, checked[i], b->done[i], checked[i], todo);
      check_list(i, todo, sp);
      const int first_new = checked[i] + 1;
      checked[i] = b->done[i];
      h->lanczos_done = b->done[i];
      LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host, h->flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, sp));
      LYAP_CUDA_TRY(cudaMemcpyAsync(h->hist_host + first_new - 1, h->hist + first_new - 1,
                                    sizeof(double) * (checked[i] - first_new + 1), cudaMemcpyDeviceToHost, sp));
      pending.push_back(i);
    }
    for (int p = 0; p < b->plan.npools; ++p) {
      cudaEventRecord(b->join[p], b->streams[p]);
      cudaStreamWaitEvent(st, b->join[p], 0);
    }
    cudaEventRecord(b->ev[3], st);
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    LYAP_CUDA_TRY(cudaGetLastError());
    cudaEventElapsedTime(&a, b->ev[2], b->ev[3]);
    t_check += a;
    if (o.check_every == LYAP_CHECK_ADAPTIVE) {
      // the adaptive schedule may have skipped m before an instance's first converged check:
      // check them, so that its m is the first converged m after its last failing check
      cudaEventRecord(b->ev[2], st);
      for (int p = 0; p < b->plan.npools; ++p) cudaStreamWaitEvent(b->streams[p], b->ev[2], 0);
      int nb = 0;
      for (int i : pending) {
        lyap_handle* h = b->h[i];
        const int mc = h->flags_host[1];
        if (mc == INT_MAX) continue;
        int last = mc - 1;
        while (last >= 1 && !was[i][last]) --last;
        todo.clear();
        for (int mm = last + 1; mm < mc; ++mm) todo.push_back(mm);
        if (todo.empty()) continue;
        cudaStream_t sp = b->streams[nb++ % b->plan.npools];
        h->check_ws = b->pool[(nb - 1) % b->plan.npools];
        check_list(i, todo, sp);
        LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host, h->flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, sp));
      }
      if (nb > 0) {
        for (int p = 0; p < b->plan.npools; ++p) {
          cudaEventRecord(b->join[p], b->streams[p]);
          cudaStreamWaitEvent(st, b->join[p], 0);
        }
        cudaEventRecord(b->ev[3], st);
        LYAP_CUDA_TRY(cudaStreamSynchronize(st));
        LYAP_CUDA_TRY(cudaGetLastError());
        cudaEventElapsedTime(&a, b->ev[2], b->ev[3]);
        t_check += a;
      }
    }
    bool stop_changed = false;
    for (int i : pending) {
      lyap_handle* h = b->h[i];
      const int rs = round_status(h);
      int fin = 0;
      if (rs != LYAP_OK) {
        b->status[i] = rs;
        b->m[i] = b->done[i];
        fin = 1;
      } else if (h->flags_host[1] != INT_MAX) {
        b->status[i] = LYAP_OK;
        b->m[i] = h->flags_host[1];
        fin = 1;
      } else if (b->done[i] >= o.maxit) {
        b->status[i] = LYAP_NOT_CONVERGED;
        b->m[i] = o.maxit;
        fin = 1;
      }
      if (fin) {
        finished[i] = 1;
        ++nfinished;
        b->h_step[2 * i + 1] = 0;
        stop_changed = true;
      }
    }
    if (stop_changed)
      LYAP_CUDA_TRY(cudaMemcpyAsync(b->d_step, b->h_step, sizeof(int) * 2 * K, cudaMemcpyHostToDevice, st));
    chunk = std::min(2 * chunk, o.check_batch);
  }
  int first_err = LYAP_OK, any_nc = 0;
  int64_t iters = 0;
  for (int i = 0; i < K; ++i) {
    rc = solve_end(b->h[i], b->done[i], b->m[i], b->status[i] == LYAP_OK ? LYAP_OK : LYAP_NOT_CONVERGED, st);
    if (rc != LYAP_OK) return rc;
    // an instance whose check failed has no usable result
    if (b->status[i] != LYAP_OK && b->status[i] != LYAP_NOT_CONVERGED) b->h[i]->solved = 0;
    iters += b->done[i];
    if (b->status[i] == LYAP_NOT_CONVERGED) any_nc = 1;
    else if (b->status[i] != LYAP_OK && first_err == LYAP_OK) first_err = b->status[i];
  }
  const int result = first_err != LYAP_OK ? first_err : (any_nc ? LYAP_NOT_CONVERGED : LYAP_OK);
  cudaEventRecord(b->ev[1], st);
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
  b->times[1] = ms;
  b->times[2] = t_lanczos;
  b->times[3] = t_check;
  b->times[4] = (double)iters;
  b->replays = replays;
  int ngroups = (int)b->groups.size();
  b->times[6] = (double)replays;
  int64_t l = b->launches + replays * 4 * ngroups;
  for (int i = 0; i < K; ++i) l += b->h[i]->launches;
  b->times[5] = (double)l;
  b->solved = 1;
  cudaStreamWaitEvent(user, b->ev[1], 0);
  return result;
}

int lyap_batch_status(lyap_batch* b, int* status, int* m) {
  if (!b || !b->solved) return LYAP_ERR_ARG;
  for (int i = 0; i < b->count; ++i) {
    if (status) status[i] = b->status[i];
    if (m) m[i] = b->m[i];
  }
  return LYAP_OK;
}

int lyap_batch_residual_norm(lyap_batch* b, int i, double* hist_host, int cap, int* m_out) {
  if (!b || i < 0 || i >= b->count || !b->solved) return LYAP_ERR_ARG;
  if (!b->h[i]->solved) {
    if (m_out) *m_out = b->m[i];
    return b->status[i];
  }
  return lyap_residual_norm(b->h[i], hist_host, cap, m_out);
}

int lyap_batch_factor(lyap_batch* b, int i, void* Z, int64_t ldz, int z_dtype, int tcap, int* t_out, void* stream) {
  if (!b || i < 0 || i >= b->count || !b->solved) return LYAP_ERR_ARG;
  lyap_handle* h = b->h[i];
  h->check_ws = b->pool[0];
  h->factor_ws = b->pool[0] + b->plan.pool_check;
  return lyap_factor(h, Z, ldz, nullptr, 0, z_dtype, LYAP_MEM_DEVICE, tcap, t_out, stream);
}

int lyap_batch_tuning(lyap_batch* b, int* out, int cap) {
  if (!b || !out) return LYAP_ERR_ARG;
  int n = 0;
  for (const Group& g : b->groups) {
    if (3 * n + 2 >= cap) break;
    out[3 * n] = g.s;
    out[3 * n + 1] = g.rows;
    out[3 * n + 2] = g.per_sm > 0 ? g.per_sm : batch_blocks_per_sm(g.s, b->opt.precision == LYAP_PREC_MIXED);
    ++n;
  }
  return n;
}

int lyap_batch_phase_times(lyap_batch* b, double* out, int cap) {
  if (!b || !out) return LYAP_ERR_ARG;
  for (int i = 0; i < cap && i < 8; ++i) out[i] = b->times[i];
  return LYAP_OK;
}

}  // extern "C"
