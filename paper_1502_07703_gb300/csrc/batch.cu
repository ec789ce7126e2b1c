// Batched form: many independent meshes of uneven sizes and degrees advanced
// together. Meshes of the same degree are stored as one disjoint-union mesh (no
// face is shared across meshes), so each RK stage is one persistent launch per
// degree over all of them; each element carries its own mesh's time step. A
// whole batch step is captured once as a CUDA graph and replayed; the degree
// groups are independent, so the graph forks them onto parallel branches (one
// stream each) and their launches of a stage run side by side, the tail of one
// overlapping the others. FP32 groups keep their face traces in a ping-pong pair
// across replays: a step flips the current half 5 x nsteps times, so two graphs
// (one per starting half) alternate and no replay re-interpolates the traces.
// For FP32 batches the elements per CTA and the persistent grid of each degree
// are autotuned at setup by timing candidates on the (all-zero) initial state,
// which leaves it unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/pyrdg.h"
#include "builder.h"
#include "handle.h"
#include "multi.h"

using pyrdg::DeviceGuard;
using pyrdg::fail;

struct pyr_dg_batch {
  int nmesh = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t tsize = 8;
  std::vector<pyr_dg*> groups;      // one union handle per degree
  std::vector<int> group_N;
  std::vector<int> mesh_group;      // group of each mesh
  std::vector<int64_t> mesh_off;    // first element of each mesh in its group
  std::vector<int64_t> mesh_K;
  std::vector<double> mesh_t;       // simulation time of each mesh
  std::vector<double> mesh_aov;     // max |dK|/|K| of each mesh
  std::vector<double> last_dt;      // per-mesh steps currently in the groups' dt_elem
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by the trace half the replay starts from
  int graph_nsteps = -1;
  std::vector<cudaStream_t> branch;  // one stream per degree group after the first (graph branches)
  std::vector<cudaEvent_t> branch_ev;  // fork event, then one join event per branch
  // single-launch mode (FP32, 2..8 groups): one kernel per stage runs every group
  bool multi = false;
  size_t multi_smem = 0;
  int multi_blocks = 0;
  pyrdg::MultiArgs margs{};
};

namespace {

void destroy_batch(pyr_dg_batch* b) {
  if (!b) return;
  for (cudaGraphExec_t& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  for (pyr_dg* h : b->groups) pyr_dg_destroy(h);
  for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->branch_ev) cudaEventDestroy(ev);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Time one step of a handle with the given elements per CTA and persistent grid (state
// must be all zero and dt_elem zero, so the step leaves it zero).
int time_grid(pyr_dg* h, int epb, int blocks, float* ms) {
  h->stage_epb = epb;
  h->stage_blocks = blocks;
  h->tr_valid = false;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(PYR_DG_ERR_CUDA, "autotune: cannot create an event");
  }
  int rc = pyrdg::enqueue_steps(h, 1, 1.0);  // warm
  if (rc == PYR_DG_OK) {
    cudaEventRecord(e0, h->stream);
    rc = pyrdg::enqueue_steps(h, 1, 1.0);
    cudaEventRecord(e1, h->stream);
  }
  const cudaError_t e = cudaEventSynchronize(e1);
  if (rc == PYR_DG_OK && e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(PYR_DG_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  return rc;
}

// Traces of the current state into half 0 of every FP32 group's ping-pong pair, when any
// group's are stale (after setup, projection or a state change); all groups then share the
// current half.
cudaError_t refresh_traces(pyr_dg_batch* b) {
  bool stale = false;
  for (pyr_dg* h : b->groups) stale = stale || (h->use_stage32 && !h->tr_valid);
  if (!stale) return cudaSuccess;
  for (pyr_dg* h : b->groups) {
    if (!h->use_stage32) continue;
    h->tr_cur = 0;
    h->L->trace(h->K, h->q, h->tab, h->tr, b->stream);
    h->tr_valid = true;
  }
  return cudaGetLastError();
}

// Enqueue nsteps steps of every mesh on the batch stream, starting from trace half `par`:
// one single-launch kernel per stage (multi mode), or each degree group on its own branch
// stream forked from and joined into the batch stream. Leaves the groups' host-side trace
// half at `par` (the caller accounts for the flips).
int enqueue_batch(pyr_dg_batch* b, int nsteps, int par, bool multi) {
  if (multi) {
    for (int n = 0; n < nsteps; ++n)
      for (int st = 0; st < 5; ++st) {
        pyrdg::multi_launch(b->margs, b->multi_blocks, b->multi_smem, (par + 5 * n + st) & 1, kRkA[st], kRkB[st],
                            b->stream);
      }
    CUDA_TRY(cudaGetLastError());
    return PYR_DG_OK;
  }
  int rc = PYR_DG_OK;
  CUDA_TRY(cudaEventRecord(b->branch_ev[0], b->stream));
  for (size_t g = 1; g < b->groups.size(); ++g) CUDA_TRY(cudaStreamWaitEvent(b->branch[g - 1], b->branch_ev[0], 0));
  for (size_t g = 0; g < b->groups.size() && rc == PYR_DG_OK; ++g) {
    pyr_dg* h = b->groups[g];
    const cudaStream_t own = h->stream;
    h->stream = g == 0 ? b->stream : b->branch[g - 1];
    h->tr_cur = par;
    rc = pyrdg::enqueue_steps(h, nsteps, 1.0);  // flips tr_cur on the host: restored below
    h->stream = own;
    h->tr_cur = par;
    h->tr_valid = true;
  }
  for (size_t g = 1; g < b->groups.size(); ++g) {
    CUDA_TRY(cudaEventRecord(b->branch_ev[g], b->branch[g - 1]));
    CUDA_TRY(cudaStreamWaitEvent(b->stream, b->branch_ev[g], 0));
  }
  return rc;
}

// Time one enqueued step of the batch in the given mode (state and dt_elem zero: unchanged).
int time_batch_step(pyr_dg_batch* b, bool multi, float* ms) {
  CUDA_TRY(refresh_traces(b));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(PYR_DG_ERR_CUDA, "autotune: cannot create an event");
  }
  int rc = enqueue_batch(b, 1, 0, multi);  // warm
  if (rc == PYR_DG_OK) {
    cudaEventRecord(e0, b->stream);
    rc = enqueue_batch(b, 1, 1, multi);
    cudaEventRecord(e1, b->stream);
  }
  const cudaError_t e = cudaEventSynchronize(e1);
  if (rc == PYR_DG_OK && e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (pyr_dg* h : b->groups) h->tr_valid = false;
  if (e != cudaSuccess) return fail(PYR_DG_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  return rc;
}

// Single-launch mode for an FP32 batch of 2..8 degree groups: upload every degree's tables to
// the multi-degree kernel, split its resident CTAs between the groups in proportion to each
// group's measured cost (its step with all CTAs on that group alone), then keep the mode only
// if a whole step is faster than the per-degree launches on graph branches.
int tune_single_launch(pyr_dg_batch* b) {
  const int ng = (int)b->groups.size();
  if (ng < 2 || ng > pyrdg::kMaxMultiGroups) return PYR_DG_OK;
  for (pyr_dg* h : b->groups)
    if (!h->use_stage32) return PYR_DG_OK;
  size_t smem = 0;
  for (pyr_dg* h : b->groups) smem = std::max(smem, pyrdg::multi_smem(h->N));
  for (pyr_dg* h : b->groups) {
    pyrdg::RefTables T;
    if (pyrdg::build_tables(h->N, T) != 0) return fail(PYR_DG_ERR_UNSUPPORTED_N, "table build failed");
    CUDA_TRY(pyrdg::multi_prepare(h->N, T.tab.data(), smem));
  }
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
  const int bps = pyrdg::multi_blocks_per_sm(smem);
  if (bps <= 0) return PYR_DG_OK;
  const int total = bps * nsm;
  b->multi_smem = smem;
  pyrdg::MultiArgs all{};
  all.ngroups = ng;
  std::vector<int64_t> egroups(ng);
  for (int g = 0; g < ng; ++g) {
    pyr_dg* h = b->groups[g];
    pyrdg::MultiGroup& G = all.g[g];
    G.N = h->N;
    G.bc = h->bc;
    G.tau = (float)h->tau;
    G.K = h->K;
    G.q = (float*)h->q;
    G.res = (float*)h->res;
    G.tr[0] = (float*)h->tr;
    G.tr[1] = (float*)h->tr2;
    G.mapP = h->mapP;
    G.geo = (const float*)h->geo;
    G.gface = (const float*)h->gface;
    G.invM = (const float*)h->invM;
    G.dt_elem = (const float*)h->dt_elem;
    const int epb = pyrdg::multi_epb_of(h->N);
    egroups[g] = (h->K + epb - 1) / epb;
  }
  // cost of each group: all CTAs (up to its element groups) on it alone
  std::vector<float> cost(ng, 0.f);
  float sum = 0.f;
  for (int g = 0; g < ng; ++g) {
    b->margs.ngroups = 1;
    b->margs.g[0] = all.g[g];
    b->margs.g[0].blk0 = 0;
    b->margs.g[0].nblk = (int)std::min<int64_t>(total, egroups[g]);
    b->multi_blocks = b->margs.g[0].nblk;
    const int rc = time_batch_step(b, true, &cost[g]);
    if (rc != PYR_DG_OK) return rc;
    sum += cost[g];
  }
  // split: proportional to cost, at least one CTA each, never more than a group's element groups
  int blk0 = 0;
  for (int g = 0; g < ng; ++g) {
    const int64_t share = (int64_t)std::llround((double)cost[g] / sum * total);
    all.g[g].blk0 = blk0;
    all.g[g].nblk = (int)std::max<int64_t>(1, std::min<int64_t>(egroups[g], share));
    blk0 += all.g[g].nblk;
  }
  b->margs = all;
  b->multi_blocks = blk0;
  float t_multi = 0.f, t_branch = 0.f;
  int rc = time_batch_step(b, true, &t_multi);
  if (rc == PYR_DG_OK) rc = time_batch_step(b, false, &t_branch);
  if (rc != PYR_DG_OK) return rc;
  b->multi = t_multi < t_branch;
  return PYR_DG_OK;
}

}  // namespace

extern "C" {

int pyr_dg_batch_setup(int nmesh, const double* const* vertices, const int64_t* Nv, const int32_t* const* EToV,
                       const int64_t* K, const int* N, const pyr_dg_opts* opts, pyr_dg_batch** out) {
  if (!out) return fail(PYR_DG_ERR_BAD_ARG, "out is null");
  *out = nullptr;
  if (nmesh < 1 || !vertices || !Nv || !EToV || !K || !N) return fail(PYR_DG_ERR_BAD_ARG, "bad batch arguments");
  pyr_dg_opts o;
  pyr_dg_default_opts(&o);
  if (opts) o = *opts;
  if (o.equation != PYR_DG_WAVE) return fail(PYR_DG_ERR_BAD_ARG, "batches hold acoustic-wave meshes only");
  if (o.basis != PYR_DG_MODAL) return fail(PYR_DG_ERR_BAD_ARG, "batches use the modal basis");
  for (int i = 0; i < nmesh; ++i) {
    if (!vertices[i] || !EToV[i] || Nv[i] < 5 || K[i] < 1)
      return fail(PYR_DG_ERR_BAD_ARG, "mesh %d: null arrays or empty sizes", i);
    if (N[i] < PYR_DG_MIN_N || N[i] > PYR_DG_MAX_N) return fail(PYR_DG_ERR_UNSUPPORTED_N, "mesh %d: N = %d", i, N[i]);
  }
  pyr_dg_batch* b = new (std::nothrow) pyr_dg_batch();
  if (!b) return fail(PYR_DG_ERR_NO_MEMORY, "host allocation failed");
  b->nmesh = nmesh;
  if (o.device >= 0) {
    b->device = o.device;
  } else if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return fail(PYR_DG_ERR_CUDA, "no CUDA device available");
  }
  DeviceGuard guard(b->device);
  if (guard.err != cudaSuccess) {
    delete b;
    return fail(PYR_DG_ERR_CUDA, "cannot select device %d", b->device);
  }
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
  } else {  // graph capture needs a stream other than the legacy default stream
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(PYR_DG_ERR_CUDA, "cannot create a stream");
    }
    b->own_stream = true;
  }
  b->tsize = o.precision == PYR_DG_F64 ? 8 : 4;
  b->mesh_group.assign(nmesh, -1);
  b->mesh_off.assign(nmesh, 0);
  b->mesh_K.assign(K, K + nmesh);
  b->mesh_t.assign(nmesh, 0.0);
  b->mesh_aov.assign(nmesh, 0.0);

  std::map<int, std::vector<int>> by_degree;
  for (int i = 0; i < nmesh; ++i) by_degree[N[i]].push_back(i);
  for (auto& kv : by_degree) {
    const int deg = kv.first;
    const std::vector<int>& ms = kv.second;
    int64_t nv_tot = 0, k_tot = 0;
    for (int i : ms) {
      nv_tot += Nv[i];
      k_tot += K[i];
    }
    if (nv_tot > 0x7fffffffLL) {
      destroy_batch(b);
      return fail(PYR_DG_ERR_BAD_ARG, "degree-%d group has too many vertices for int32 indexing", deg);
    }
    std::vector<double> V((size_t)nv_tot * 3);
    std::vector<int32_t> E((size_t)k_tot * 5);
    int64_t voff = 0, eoff = 0;
    std::vector<double> xg(deg + 1), wg(deg + 1);
    pyrdg::gauss_jacobi(deg + 1, 0.0, 0.0, xg.data(), wg.data());
    for (int i : ms) {
      std::memcpy(&V[(size_t)voff * 3], vertices[i], (size_t)Nv[i] * 3 * sizeof(double));
      double aov = 0.0;
      for (int64_t e = 0; e < K[i]; ++e) {
        double v15[15];
        for (int c = 0; c < 5; ++c) {
          const int32_t vi = EToV[i][e * 5 + c];
          if (vi < 0 || vi >= Nv[i]) {
            destroy_batch(b);
            return fail(PYR_DG_ERR_BAD_MESH, "mesh %d: EToV[%lld][%d] = %d out of range", i, (long long)e, c, vi);
          }
          E[(size_t)(eoff + e) * 5 + c] = (int32_t)(vi + voff);
          for (int m = 0; m < 3; ++m) v15[c * 3 + m] = vertices[i][(int64_t)vi * 3 + m];
        }
        aov = std::max(aov, pyrdg::area_over_volume(v15, xg.data(), wg.data(), deg + 1));
      }
      b->mesh_group[i] = (int)b->groups.size();
      b->mesh_off[i] = eoff;
      b->mesh_aov[i] = aov;
      voff += Nv[i];
      eoff += K[i];
    }
    pyr_dg_opts go = o;
    go.stream = b->stream;
    go.device = b->device;
    pyr_dg* h = nullptr;
    const int rc = pyr_dg_setup(V.data(), nv_tot, E.data(), k_tot, deg, &go, &h);
    if (rc != PYR_DG_OK) {
      destroy_batch(b);
      return rc;  // message already set
    }
    b->groups.push_back(h);
    b->group_N.push_back(deg);
    if (cudaMalloc(&h->dt_elem, (size_t)k_tot * b->tsize) != cudaSuccess ||
        cudaMemsetAsync(h->dt_elem, 0, (size_t)k_tot * b->tsize, b->stream) != cudaSuccess) {
      destroy_batch(b);
      return fail(PYR_DG_ERR_NO_MEMORY, "cannot allocate the per-element time steps");
    }
    // Autotune the FP32 stage kernel on the zero state: elements per CTA (1, 2, 4, 8 where
    // built for this degree) and the persistent grid (1 .. resident CTAs per SM, per SM).
    if (h->use_stage32 && h->K >= 4096) {
      int nsm = 1;
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
      int best_epb = h->stage_epb, best = h->stage_blocks;
      float best_ms = 1e30f;
      const int epbs[] = {1, 2, 4, 8};
      for (int epb : epbs) {
        const int bps = h->L->blocks_per_sm32(epb);
        if (bps <= 0) continue;
        const int64_t groups = (h->K + epb - 1) / epb;
        for (int m = 1; m <= bps; ++m) {
          const int blocks = (int)std::min<int64_t>(groups, (int64_t)m * nsm);
          float ms = 0.f;
          const int trc = time_grid(h, epb, blocks, &ms);
          if (trc != PYR_DG_OK) {
            destroy_batch(b);
            return trc;
          }
          if (ms < best_ms) {
            best_ms = ms;
            best_epb = epb;
            best = blocks;
          }
        }
      }
      h->stage_epb = best_epb;
      h->stage_blocks = best;
      h->tr_valid = false;
    }
  }
  // graph branches: a stream per further degree group, a fork event and a join event per branch
  for (size_t g = 1; g < b->groups.size(); ++g) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      destroy_batch(b);
      return fail(PYR_DG_ERR_CUDA, "cannot create a branch stream");
    }
    b->branch.push_back(st);
  }
  for (size_t g = 0; g < b->groups.size(); ++g) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      destroy_batch(b);
      return fail(PYR_DG_ERR_CUDA, "cannot create a branch event");
    }
    b->branch_ev.push_back(ev);
  }
  {
    const int trc = tune_single_launch(b);
    if (trc != PYR_DG_OK) {
      destroy_batch(b);
      return trc;
    }
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    destroy_batch(b);
    return fail(PYR_DG_ERR_CUDA, "batch setup failed");
  }
  *out = b;
  return PYR_DG_OK;
}

int pyr_dg_batch_info(const pyr_dg_batch* b, int* nmesh, int* ngroups, int64_t* total_K, int64_t* total_dofs) {
  if (!b) return fail(PYR_DG_ERR_BAD_ARG, "null batch");
  int64_t tk = 0, td = 0;
  for (const pyr_dg* h : b->groups) {
    tk += h->K;
    td += h->K * 4 * h->Np;
  }
  if (nmesh) *nmesh = b->nmesh;
  if (ngroups) *ngroups = (int)b->groups.size();
  if (total_K) *total_K = tk;
  if (total_dofs) *total_dofs = td;
  return PYR_DG_OK;
}

int pyr_dg_batch_group_info(const pyr_dg_batch* b, int group, int* N, int64_t* K, int* stage_blocks,
                            int* elems_per_block) {
  if (!b || group < 0 || group >= (int)b->groups.size()) return fail(PYR_DG_ERR_BAD_ARG, "bad group");
  const pyr_dg* h = b->groups[group];
  if (N) *N = h->N;
  if (K) *K = h->K;
  if (b->multi) {  // the group's CTAs of the single-launch kernel
    if (stage_blocks) *stage_blocks = b->margs.g[group].nblk;
    if (elems_per_block) *elems_per_block = pyrdg::multi_epb_of(h->N);
    return PYR_DG_OK;
  }
  if (stage_blocks) *stage_blocks = h->use_stage32 ? h->stage_blocks : (int)h->K;
  if (elems_per_block) *elems_per_block = h->use_stage32 ? h->stage_epb : 1;
  return PYR_DG_OK;
}

int pyr_dg_batch_set_launch_mode(pyr_dg_batch* b, int single_launch) {
  if (!b) return fail(PYR_DG_ERR_BAD_ARG, "null batch");
  if (single_launch && b->multi_blocks <= 0)
    return fail(PYR_DG_ERR_BAD_ARG, "the single-launch stage needs an FP32 batch of 2 to %d degree groups",
                pyrdg::kMaxMultiGroups);
  if ((single_launch != 0) != b->multi) {
    DeviceGuard g(b->device);
    CUDA_TRY(g.err);
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (cudaGraphExec_t& gx : b->graph)
      if (gx) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
      }
    b->multi = single_launch != 0;
  }
  return PYR_DG_OK;
}

int pyr_dg_batch_launch_mode(const pyr_dg_batch* b, int* single_launch, int* launches_per_stage) {
  if (!b) return fail(PYR_DG_ERR_BAD_ARG, "null batch");
  if (single_launch) *single_launch = b->multi ? 1 : 0;
  if (launches_per_stage) *launches_per_stage = b->multi ? 1 : (int)b->groups.size();
  return PYR_DG_OK;
}

int pyr_dg_batch_project(pyr_dg_batch* b, double t0) {
  if (!b) return fail(PYR_DG_ERR_BAD_ARG, "null batch");
  for (pyr_dg* h : b->groups) {
    const int rc = pyr_dg_project(h, t0);
    if (rc != PYR_DG_OK) return rc;
  }
  std::fill(b->mesh_t.begin(), b->mesh_t.end(), t0);
  return PYR_DG_OK;
}

int pyr_dg_batch_dt_cfl(const pyr_dg_batch* b, double cfl, double* dt) {
  if (!b || !dt || !(cfl > 0.0)) return fail(PYR_DG_ERR_BAD_ARG, "bad arguments");
  for (int i = 0; i < b->nmesh; ++i) {
    const int n = b->group_N[b->mesh_group[i]];
    const double CN = 2.0 * (n + 1) * (n + 3) / 3.0;
    dt[i] = cfl / (CN * b->mesh_aov[i]);
  }
  return PYR_DG_OK;
}

int pyr_dg_batch_step(pyr_dg_batch* b, int nsteps, const double* dt) {
  if (!b || !dt) return fail(PYR_DG_ERR_BAD_ARG, "null argument");
  if (nsteps < 0) return fail(PYR_DG_ERR_BAD_ARG, "nsteps must be >= 0");
  for (int i = 0; i < b->nmesh; ++i)
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(PYR_DG_ERR_BAD_ARG, "dt[%d] must be > 0", i);
  if (nsteps == 0) return PYR_DG_OK;
  DeviceGuard g(b->device);
  CUDA_TRY(g.err);
  // per-element steps, uploaded only when they change
  if (b->last_dt.size() != (size_t)b->nmesh || !std::equal(b->last_dt.begin(), b->last_dt.end(), dt)) {
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      pyr_dg* h = b->groups[gi];
      std::vector<double> d64;
      std::vector<float> d32;
      if (b->tsize == 8)
        d64.assign((size_t)h->K, 0.0);
      else
        d32.assign((size_t)h->K, 0.f);
      for (int i = 0; i < b->nmesh; ++i) {
        if (b->mesh_group[i] != (int)gi) continue;
        for (int64_t e = 0; e < b->mesh_K[i]; ++e) {
          if (b->tsize == 8)
            d64[(size_t)(b->mesh_off[i] + e)] = dt[i];
          else
            d32[(size_t)(b->mesh_off[i] + e)] = (float)dt[i];
        }
      }
      const void* src = b->tsize == 8 ? (const void*)d64.data() : (const void*)d32.data();
      CUDA_TRY(cudaMemcpyAsync(h->dt_elem, src, (size_t)h->K * b->tsize, cudaMemcpyHostToDevice, b->stream));
      CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    b->last_dt.assign(dt, dt + b->nmesh);
  }
  if (b->graph_nsteps != nsteps) {
    for (cudaGraphExec_t& gx : b->graph)
      if (gx) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
      }
    b->graph_nsteps = nsteps;
  }
  CUDA_TRY(refresh_traces(b));
  int par = 0;
  for (pyr_dg* h : b->groups)
    if (h->use_stage32) par = h->tr_cur;
  if (!b->graph[par]) {
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_batch(b, nsteps, par, b->multi);
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
    if (rc != PYR_DG_OK || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (rc != PYR_DG_OK) return rc;
      return fail(PYR_DG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ee));
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->graph[par], graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(PYR_DG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  }
  CUDA_TRY(cudaGraphLaunch(b->graph[par], b->stream));
  for (pyr_dg* h : b->groups)
    if (h->use_stage32) h->tr_cur = (h->tr_cur + 5 * nsteps) & 1;  // the half the replay ended in
  for (int i = 0; i < b->nmesh; ++i) b->mesh_t[i] += nsteps * dt[i];
  return PYR_DG_OK;
}

int pyr_dg_batch_error(pyr_dg_batch* b, double* l2_abs, double* l2_rel) {
  if (!b) return fail(PYR_DG_ERR_BAD_ARG, "null batch");
  DeviceGuard g(b->device);
  CUDA_TRY(g.err);
  for (int i = 0; i < b->nmesh; ++i) {
    pyr_dg* h = b->groups[b->mesh_group[i]];
    const int64_t off = b->mesh_off[i], Ki = b->mesh_K[i];
    const int nb = (int)std::min<int64_t>(Ki, h->err_blocks);
    const char* q = (const char*)h->q + (size_t)off * 4 * h->Np * h->tsize;
    h->L->error(Ki, q, h->ev + off * 15, h->gtab, h->bc, b->mesh_t[i], h->partial, nb, b->stream);
    CUDA_TRY(cudaGetLastError());
    std::vector<double> part((size_t)nb * 2);
    CUDA_TRY(cudaMemcpyAsync(part.data(), h->partial, part.size() * 8, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    double e2 = 0.0, n2 = 0.0;
    for (int k = 0; k < nb; ++k) {
      e2 += part[2 * k];
      n2 += part[2 * k + 1];
    }
    if (l2_abs) l2_abs[i] = std::sqrt(e2);
    if (l2_rel) l2_rel[i] = n2 > 0 ? std::sqrt(e2 / n2) : std::sqrt(e2);
  }
  return PYR_DG_OK;
}

int pyr_dg_batch_get_state(pyr_dg_batch* b, int mesh, void* q, int where) {
  if (!b || !q || mesh < 0 || mesh >= b->nmesh) return fail(PYR_DG_ERR_BAD_ARG, "bad arguments");
  if (where != PYR_DG_HOST && where != PYR_DG_DEVICE) return fail(PYR_DG_ERR_BAD_ARG, "bad `where`");
  DeviceGuard g(b->device);
  CUDA_TRY(g.err);
  pyr_dg* h = b->groups[b->mesh_group[mesh]];
  const size_t per = (size_t)4 * h->Np * h->tsize;
  CUDA_TRY(cudaMemcpyAsync(q, (const char*)h->q + b->mesh_off[mesh] * per, b->mesh_K[mesh] * per,
                           where == PYR_DG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PYR_DG_OK;
}

int pyr_dg_batch_sync(pyr_dg_batch* b) {
  if (!b) return fail(PYR_DG_ERR_BAD_ARG, "null batch");
  DeviceGuard g(b->device);
  CUDA_TRY(g.err);
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PYR_DG_OK;
}

void* pyr_dg_batch_stream(const pyr_dg_batch* b) { return b ? (void*)b->stream : nullptr; }

void pyr_dg_batch_destroy(pyr_dg_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  destroy_batch(b);
}

}  // extern "C"
