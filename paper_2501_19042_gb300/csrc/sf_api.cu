// Host side of the C ABI declared in include/sf.h: argument validation,
// handle lifetime, work decomposition of a batch into launches, and the
// device-status word.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "sf_debug.cuh"
#include "sf_internal.cuh"

struct sf_handle {
  sf_problem pb;
  int device = 0;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  float* basis = nullptr;   // [T][BASIS_ROW]
  float* ops = nullptr;     // [max_robots + 1][OPS_STRIDE]
  int* status = nullptr;    // device status word
  unsigned long long launches = 0;
  int force_G = 0, force_warps = 0, force_tc = 0;  // launch-shape overrides (tuning)
  int last_plan[4] = {0, 0, 0, 0};                 // G, warps, tc, nq of the last fused launch
  int last_form = 0;                               // its form: 1 tensor memory, 0 float32 lanes
  std::map<std::string, sf::FusedPlan> tuned;      // autotuned shapes per launch-group key
  bool use_tuned = true;
  int prune = 1;                                   // SF_OPT_PAIR_PRUNING
  int tm = 2;                                      // SF_OPT_TENSOR_MEMORY (2: per bucket)
  int wait_test_us = 0;                            // SF_OPT_TEST_WAIT_TIMEOUT
  int plant_canary = 0;                            // SF_OPT_TEST_CANARY (debug builds)
  cudaStream_t aux[2] = {nullptr, nullptr};        // extra streams for concurrent launch groups
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  float eq_pi[sf::NV * sf::NV] = {};               // QP layer operators (host copy of slot 0)
  float eq_r[sf::NV * 6] = {};
  std::string err;
};

namespace {

using namespace sf;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

sf_status fail(sf_handle* h, sf_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

const char* debug_site_name(int site) {
  switch (site) {
    case sf::DS_PAIR_DECODE: return "pair decoded from a candidate bit";
    case sf::DS_CHUNK_ROW: return "chunk-buffer row";
    case sf::DS_TMEM_COL: return "TMEM column";
    case sf::DS_TABLE: return "MMA B-table word";
    case sf::DS_MASK: return "activity-mask word";
    case sf::DS_OUT: return "global output index";
    case sf::DS_CANARY_HEAD: return "canary after the shared-memory head";
    case sf::DS_CANARY_BLOCK: return "canary at the end of a sample block";
    default: return "unknown site";
  }
}

sf_status cuda_fail(sf_handle* h, cudaError_t e, const char* where) {
  return fail(h, SF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int bucket_index(int N) { return N <= 8 ? 0 : (N <= 16 ? 1 : (N <= 24 ? 2 : 3)); }
constexpr int kBuckets = 4;
constexpr int kBucketNmax[kBuckets] = {8, 16, 24, 32};

ProblemConsts consts(const sf_problem& pb, int K) {
  ProblemConsts c;
  c.dim = pb.dim;
  c.T = pb.T;
  c.K = K;
  c.rho = (float)pb.rho;
  c.inv_a2 = (float)(1.0 / (pb.coll_a * pb.coll_a));
  c.inv_b2 = (float)(1.0 / (pb.coll_b * pb.coll_b));
  c.inv_a = (float)(1.0 / pb.coll_a);
  c.inv_b = (float)(1.0 / pb.coll_b);
  c.coll_a = (float)pb.coll_a;
  c.coll_b = (float)pb.coll_b;
  c.tie = (float)(pb.dim == 3 ? pb.coll_b : pb.coll_a);
  c.use_v = pb.v_max > 0.0;
  c.use_a = pb.a_max > 0.0;
  c.v_max = (float)(c.use_v ? pb.v_max : 0.0);
  c.a_max = (float)(c.use_a ? pb.a_max : 0.0);
  c.use_w = pb.use_workspace ? 1 : 0;
  for (int x = 0; x < 3; ++x) {
    const double wa = x == 2 ? pb.ws_b : pb.ws_a;
    const double ca = x == 2 ? pb.coll_b : pb.coll_a;
    c.wc[x] = c.use_w ? (float)pb.ws_center[x] : 0.0f;
    c.wa[x] = c.use_w ? (float)wa : 0.0f;
    c.winv[x] = c.use_w ? (float)(1.0 / wa) : 0.0f;
    c.wk[x] = c.use_w ? (float)(ca / wa) : 0.0f;
    c.wo[x] = c.use_w ? (float)(pb.ws_center[x] / wa) : 0.0f;
  }
  return c;
}

sf_status check_batch(sf_handle* h, const sf_batch* b, long long* tot_robots, long long* tot_samples) {
  if (!b) return fail(h, SF_ERR_INVALID_ARG, "batch is NULL");
  if (b->n_scenes < 1 || b->n_scenes > SF_MAX_SCENES)
    return fail(h, SF_ERR_INVALID_ARG, "n_scenes out of range");
  if (!b->n_robots || !b->n_samples) return fail(h, SF_ERR_INVALID_ARG, "n_robots / n_samples is NULL");
  long long R = 0, S = 0;
  for (int s = 0; s < b->n_scenes; ++s) {
    const int N = b->n_robots[s], Ss = b->n_samples[s];
    if (N < 1 || N > h->pb.max_robots)
      return fail(h, SF_ERR_INVALID_ARG, "scene " + std::to_string(s) + ": n_robots outside 1..max_robots");
    if (Ss < 0) return fail(h, SF_ERR_INVALID_ARG, "scene " + std::to_string(s) + ": negative n_samples");
    R += N;
    S += Ss;
  }
  if (!b->start || !b->goal) return fail(h, SF_ERR_INVALID_ARG, "start / goal is NULL");
  if (S > 0 && !b->xi_bar) return fail(h, SF_ERR_INVALID_ARG, "xi_bar is NULL");
  if (S > (1LL << 30)) return fail(h, SF_ERR_INVALID_ARG, "too many samples");
  *tot_robots = R;
  *tot_samples = S;
  return SF_OK;
}


struct FusedRequest {
  const float* xi0 = nullptr;
  const float* lam0 = nullptr;
  float* xi_out = nullptr;
  float* lam_out = nullptr;
  float* resid_out = nullptr;
  float* hist = nullptr;
  float* ckpt = nullptr;
  float* fp_res2 = nullptr;
  bool backward = false;
  int prec = 0;             // forward only: the form code (FusedLaunch::prec)
  BwdLaunchArgs bwd{};
};

// Form code of a fused forward launch (FusedLaunch::prec): the tensor-memory
// form with the handle's operand format when the option is on or the
// precision is 16-bit (the 16-bit products exist only there), the float32
// form when the option is off, and FORM_AUTO (float32 handles, option 2, the
// default) to let each launch group take the form measured faster for its
// dimension, robot-count bucket and launch shape (auto_tm_candidate,
// kAutoTmMinLanes). The training forward follows
// the same rule; the adjoint is the float32 form's in every case.
constexpr int FORM_AUTO = -1;
int forward_form(const sf_handle* h) {
  const int p = h->pb.precision;
  if (p != SF_PREC_FP32 || h->tm == 1) return PREC_TM_TF32 + p;
  return h->tm == 0 ? 0 : FORM_AUTO;
}
// The float32 handle's form for one launch group under FORM_AUTO: the
// tensor-memory form where it measured faster than the float32 form on a
// GB300, i.e. 3D scenes of 9..24 robots whose tensor-memory launch shape uses
// at least 96 of the 128 TMEM lanes of a CTA (G x NMAX >= 96: 6 samples per
// CTA at 9..16 robots, 4 at 17..24). Measured, T = 100: 16 robots, 768..2048
// samples 0.67..0.69x the float32 form's time at K = 200 and 0.83..0.86x at
// K = 50, 512 samples (4 per CTA) 0.93x / 1.07x, <= 256 samples 1.2..1.4x;
// 12 robots, 1024 samples 0.66x; 20 and 24 robots, 1024 samples 0.83x and
// 0.88x; 4, 8, 28, 32 robots and every 2D case slower.
bool auto_tm_candidate(int dim, int nmax) { return dim == 3 && (nmax == 16 || nmax == 24); }
constexpr int kAutoTmMinLanes = 96;

long long total_coefs(const sf_handle* h, const sf_batch* b) {
  long long c = 0;
  for (int q = 0; q < b->n_scenes; ++q) c += (long long)b->n_samples[q] * h->pb.dim * b->n_robots[q] * NV;
  return c;
}

// Words of one activity-mask slot (one iteration of every sample): per
// sample and time step a row of mask_words(bucket N_max) words.
long long mask_slot_words(const sf_handle* h, const sf_batch* b) {
  long long w = 0;
  for (int q = 0; q < b->n_scenes; ++q)
    w += (long long)b->n_samples[q] * h->pb.T * mask_words(kBucketNmax[bucket_index(b->n_robots[q])]);
  return w;
}

// Floats of a buffer of `n_states` (xi, lambda) states, rounded up to 16 bytes
// (the activity masks follow it).
long long states_floats_aligned(long long n_states, long long coefs) { return (n_states * 2 * coefs + 3) / 4 * 4; }

struct LaunchGroup {
  FusedArgs a;
  FusedLaunch l;
  std::string key;
};

std::string group_key(bool bwd, int prec, int dim, int nmax, int T, const std::vector<int>& nr,
                      const std::vector<int>& ns) {
  std::string k = (bwd ? "b" : "f") + std::to_string(prec) + "/" + std::to_string(dim) + "/" + std::to_string(nmax) +
                  "/" + std::to_string(T) + ":";
  for (size_t q = 0; q < nr.size(); ++q) k += std::to_string(nr[q]) + "x" + std::to_string(ns[q]) + ",";
  return k;
}

// Fused form: scenes grouped by robot-count bucket, one launch per group of
// up to MAX_SCENES_PER_LAUNCH scenes. The launch shape is the autotuned one
// for the group's key when known, else the planner's.
sf_status build_groups(sf_handle* h, const sf_batch* b, int K, long long S, const FusedRequest& rq,
                       std::vector<LaunchGroup>* out) {
  const int dim = h->pb.dim, T = h->pb.T;
  const ProblemConsts pc = consts(h->pb, K);
  const long long tot = total_coefs(h, b);
  struct Item { int scene; long long roff, soff, coff, moff; };
  std::vector<Item> items[kBuckets];
  {
    long long roff = 0, soff = 0, coff = 0, moff = 0;
    for (int sc = 0; sc < b->n_scenes; ++sc) {
      const int N = b->n_robots[sc], Ss = b->n_samples[sc];
      const int bk = bucket_index(N);
      if (Ss > 0) items[bk].push_back({sc, roff, soff, coff, moff});
      roff += N;
      soff += Ss;
      coff += (long long)Ss * dim * N * NV;
      moff += (long long)Ss * T * mask_words(kBucketNmax[bk]);
    }
  }
  // longest processing time first: a CTA's work grows with its scene's robot
  // count (N (N - 1) / 2 pair rows per step), and the block scheduler starts
  // CTAs in index order as SMs free up, so the scenes of a launch are laid
  // out by decreasing N (the outputs keep the batch's own layout)
  for (int bk = 0; bk < kBuckets; ++bk)
    std::stable_sort(items[bk].begin(), items[bk].end(),
                     [&](const Item& x, const Item& y) { return b->n_robots[x.scene] > b->n_robots[y.scene]; });
  for (int bk = 0; bk < kBuckets; ++bk) {
    const int nmax = kBucketNmax[bk];
    const bool auto_tm = !rq.backward && rq.prec == FORM_AUTO && auto_tm_candidate(dim, nmax);
    const int prec0 = rq.backward ? 0 : rq.prec == FORM_AUTO ? (auto_tm ? PREC_TM_TF32 : 0) : rq.prec;
    for (size_t first = 0; first < items[bk].size(); first += MAX_SCENES_PER_LAUNCH) {
      const size_t last = std::min(items[bk].size(), first + (size_t)MAX_SCENES_PER_LAUNCH);
      std::vector<int> nr, ns;
      for (size_t q = first; q < last; ++q) {
        nr.push_back(b->n_robots[items[bk][q].scene]);
        ns.push_back(b->n_samples[items[bk][q].scene]);
      }
      LaunchGroup lg;
      const bool forced = h->force_G || h->force_warps || h->force_tc;
      auto make_plan = [&](int pr, std::string* key) {
        *key = group_key(rq.backward, pr, dim, nmax, T, nr, ns);
        auto hit = h->tuned.find(*key);
        if (!forced && h->use_tuned && hit != h->tuned.end()) return hit->second;
        return plan_fused(dim, nmax, T, nr.data(), ns.data(), (int)nr.size(), h->num_sms, h->max_smem_optin,
                          h->force_G, h->force_warps, h->force_tc, rq.backward, nullptr, 0, pr);
      };
      int prec = prec0;
      FusedPlan plan = make_plan(prec, &lg.key);
      if (auto_tm && plan.G * nmax < kAutoTmMinLanes) {   // too few rows per CTA: the float32 form
        prec = 0;
        plan = make_plan(prec, &lg.key);
      }
      if (plan.G == 0) return fail(h, SF_ERR_UNSUPPORTED, "no fused launch shape fits in shared memory");
      FusedArgs& a = lg.a;
      std::memset(&a, 0, sizeof(a));
      a.pc = pc;
      a.basis = reinterpret_cast<const float4*>(h->basis);
      a.ops = h->ops;
      a.start = b->start;
      a.goal = b->goal;
      a.start_va = b->start_va;
      a.goal_va = b->goal_va;
      a.xi_bar = b->xi_bar;
      a.xi0 = rq.xi0;
      a.lam0 = rq.lam0;
      a.xi_out = rq.xi_out;
      a.lam_out = rq.lam_out;
      a.resid_out = rq.resid_out;
      a.hist = rq.hist;
      a.total_samples = (int)S;
      a.status = h->status;
      a.tc = plan.tc;
      a.nq = plan.nq;
      a.ckpt = rq.ckpt;
      a.ck_every = std::max(1, h->pb.checkpoint_every);
      a.total_coefs = tot;
      a.fp_res2 = rq.fp_res2;
      a.prune = h->prune ? 1 : 0;
      a.wait_ns = 1000ull * (unsigned long long)h->wait_test_us;
      a.skip_first_mma = h->wait_test_us > 0 ? 1 : 0;
      a.dbg_plant = h->plant_canary;
      if (rq.ckpt && !rq.backward) {
        const long long ck = a.ck_every, nck = (K + ck - 1) / ck;
        a.amask = reinterpret_cast<unsigned*>(rq.ckpt + states_floats_aligned(nck + ck + 1, tot));
        a.amask_slot = mask_slot_words(h, b);
      }
      int ctas = 0, gmax = 1;
      a.n_scenes = (int)(last - first);
      for (size_t q = first; q < last; ++q) {
        const Item& it = items[bk][q];
        SceneDesc& d = a.sc[q - first];
        d.N = b->n_robots[it.scene];
        d.S = b->n_samples[it.scene];
        d.G = std::min(plan.G, d.S);
        d.cta_begin = ctas;
        d.robot_off = (int)it.roff;
        d.sample_off = (int)it.soff;
        d.coef_off = it.coff;
        d.mask_off = it.moff;
        ctas += (d.S + d.G - 1) / d.G;
        gmax = std::max(gmax, d.G);
      }
      FusedLaunch& l = lg.l;
      l.nmax = nmax;
      l.gmax = gmax;
      l.n_ctas = ctas;
      l.warps = plan.warps;
      l.tc = plan.tc;
      l.nq = plan.nq;
      l.prec = prec;
      l.smem = fused_smem_bytes(dim, nmax, T, gmax, plan.tc, plan.nq, rq.backward, prec);
      if (l.smem > h->max_smem_optin) return fail(h, SF_ERR_UNSUPPORTED, "launch shape exceeds shared memory");
      h->last_plan[0] = plan.G;
      h->last_plan[1] = plan.warps;
      h->last_plan[2] = plan.tc;
      h->last_plan[3] = plan.nq;
      h->last_form = (!rq.backward && prec >= PREC_TM_TF32) ? 1 : 0;
      out->push_back(lg);
    }
  }
  return SF_OK;
}

cudaError_t launch_group(const LaunchGroup& g, const FusedRequest& rq, cudaStream_t st) {
  return rq.backward ? launch_backward(g.a, rq.bwd, g.l, st) : launch_fused(g.a, g.l, st);
}

// Launches the groups; with more than one group they run concurrently on
// the handle's extra streams, forked from and joined back to `st` (inside a
// stream capture this becomes parallel branches of the graph).
sf_status launch_groups(sf_handle* h, cudaStream_t st, const std::vector<LaunchGroup>& gs, const FusedRequest& rq) {
  const char* what = rq.backward ? "backward launch" : "fused form launch";
  if (gs.size() == 1) {
    cudaError_t e = launch_group(gs[0], rq, st);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    h->launches += 1;
    return SF_OK;
  }
  cudaError_t e = cudaEventRecord(h->fork, st);
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(h->aux[q], h->fork, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "fork of launch groups");
  // up to 3 groups at once: longest first, each onto the stream with the
  // least work so far (work of a group ~ sum over its scenes of S (N^2 + 8 N))
  std::vector<double> cost(gs.size(), 0.0);
  std::vector<size_t> order(gs.size());
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    order[gi] = gi;
    for (int q = 0; q < gs[gi].a.n_scenes; ++q) {
      const double N = gs[gi].a.sc[q].N;
      cost[gi] += (double)gs[gi].a.sc[q].S * (N * N + 8.0 * N);
    }
  }
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  double load[3] = {0.0, 0.0, 0.0};
  for (size_t gi : order) {
    int q = 0;
    for (int r = 1; r < 3; ++r)
      if (load[r] < load[q]) q = r;
    load[q] += cost[gi];
    e = launch_group(gs[gi], rq, q == 0 ? st : h->aux[q - 1]);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    h->launches += 1;
  }
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    e = cudaEventRecord(h->join[q], h->aux[q]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->join[q], 0);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "join of launch groups");
  return SF_OK;
}

sf_status run_fused(sf_handle* h, cudaStream_t st, const sf_batch* b, int K, long long S, const FusedRequest& rq) {
  std::vector<LaunchGroup> gs;
  sf_status s = build_groups(h, b, K, S, rq, &gs);
  if (s != SF_OK) return s;
  return launch_groups(h, st, gs, rq);
}

}  // namespace

extern "C" {

sf_status sf_create(const sf_problem* pb, int device, sf_handle** out) {
  if (!out) return SF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!pb) return SF_ERR_INVALID_ARG;
  if (pb->dim != 2 && pb->dim != 3) return SF_ERR_INVALID_ARG;
  if (pb->order != 10) return SF_ERR_UNSUPPORTED;  // kernels are built for nvar = 11
  if (pb->T < 2 || pb->T > SF_MAX_T) return SF_ERR_INVALID_ARG;
  if (!finite_pos(pb->t_final) || !finite_pos(pb->rho) || !finite_pos(pb->coll_a) ||
      !finite_pos(pb->coll_b))
    return SF_ERR_INVALID_ARG;
  if (!std::isfinite(pb->v_max) || !std::isfinite(pb->a_max)) return SF_ERR_INVALID_ARG;
  if (pb->max_robots < 1 || pb->max_robots > SF_MAX_ROBOTS) return SF_ERR_INVALID_ARG;
  if (pb->precision < SF_PREC_FP32 || pb->precision > SF_PREC_FP16) return SF_ERR_INVALID_ARG;
  if (pb->checkpoint_every < 0) return SF_ERR_INVALID_ARG;
  if (pb->use_workspace != 0 && pb->use_workspace != 1) return SF_ERR_INVALID_ARG;
  if (pb->use_workspace) {
    if (!finite_pos(pb->ws_a) || !finite_pos(pb->ws_b)) return SF_ERR_INVALID_ARG;
    for (int x = 0; x < 3; ++x)
      if (!std::isfinite(pb->ws_center[x])) return SF_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SF_ERR_CUDA;

  sf_handle* h = new (std::nothrow) sf_handle();
  if (!h) return SF_ERR_OOM;
  h->pb = *pb;
  h->device = device;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete h; return SF_ERR_CUDA; }
  h->num_sms = prop.multiProcessorCount;
  // (debug builds: room for the static debug word of every fused kernel)
  h->max_smem_optin = prop.sharedMemPerBlockOptin - (SF_DEBUG_CHECKS ? 16 : 0);
  double* scratch = nullptr;
  const size_t nscr = precompute_scratch_doubles(pb->T, pb->order, pb->max_robots);
  cudaError_t e = cudaMalloc(&h->basis, sizeof(float) * (size_t)pb->T * BASIS_ROW);
  if (e == cudaSuccess) e = cudaMalloc(&h->ops, sizeof(float) * (size_t)(pb->max_robots + 1) * OPS_STRIDE);
  if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&scratch, sizeof(double) * nscr);
  if (e != cudaSuccess) {
    cudaFree(scratch);
    sf_destroy(h);
    return SF_ERR_OOM;
  }
  cudaStream_t st;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    e = cudaMemsetAsync(h->status, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = launch_precompute(pb->T, pb->order, pb->t_final, pb->rho, pb->v_max > 0, pb->a_max > 0,
                            pb->use_workspace, pb->max_robots, h->basis, h->ops, scratch, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(scratch);
  if (e != cudaSuccess) {
    sf_destroy(h);
    return e == cudaErrorInvalidValue ? SF_ERR_INVALID_ARG : SF_ERR_CUDA;
  }
  {
    // host copy of the QP layer's operators (slot 0), passed as kernel parameters
    std::vector<float> slot(OPS_STRIDE);
    e = cudaMemcpy(slot.data(), h->ops, sizeof(float) * OPS_STRIDE, cudaMemcpyDeviceToHost);
    for (int r = 0; r < NV && e == cudaSuccess; ++r) {
      for (int c = 0; c < NV; ++c) h->eq_pi[r * NV + c] = slot[OPS_S1 + r * NP + c];
      for (int q = 0; q < 6; ++q) h->eq_r[r * 6 + q] = slot[OPS_R1 + r * 8 + q];
    }
  }
  if (e == cudaSuccess) e = prepare_kernels(pb->dim, (int)h->max_smem_optin, pb->precision);
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    e = cudaStreamCreateWithFlags(&h->aux[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    sf_destroy(h);
    return SF_ERR_CUDA;
  }
  *out = h;
  return SF_OK;
}

void sf_destroy(sf_handle* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  for (int q = 0; q < 2; ++q) {
    if (h->aux[q]) cudaStreamDestroy(h->aux[q]);
    if (h->join[q]) cudaEventDestroy(h->join[q]);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  cudaFree(h->basis);
  cudaFree(h->ops);
  cudaFree(h->status);
  delete h;
}

const char* sf_last_error(const sf_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

size_t sf_workspace_bytes(const sf_handle* hc, const sf_batch* b, int form, int K) {
  sf_handle* h = const_cast<sf_handle*>(hc);
  if (!h) return 0;
  long long R = 0, S = 0;
  if (check_batch(h, b, &R, &S) != SF_OK) return 0;
  if (K < 1) return 0;
  if (form == SF_FORM_FUSED) return 0;
  if (form != SF_FORM_PLAIN) return 0;
  size_t best = 0;
  for (int s = 0; s < b->n_scenes; ++s)
    best = std::max(best, plain_workspace_floats(h->pb.dim, b->n_robots[s], b->n_samples[s], h->pb.T));
  return best * sizeof(float) + 256;
}

size_t sf_checkpoint_bytes(const sf_handle* hc, const sf_batch* b, int K) {
  sf_handle* h = const_cast<sf_handle*>(hc);
  if (!h || h->pb.checkpoint_every <= 0 || K < 1) return 0;
  long long R = 0, S = 0;
  if (check_batch(h, b, &R, &S) != SF_OK) return 0;
  const long long ck = h->pb.checkpoint_every;
  const long long nck = (K + ck - 1) / ck;
  // checkpoints, the iterates of the last segment (up to checkpoint_every + 1),
  // then the activity masks of the last segment's iterations
  return (size_t)(states_floats_aligned(nck + ck + 1, total_coefs(h, b)) + ck * mask_slot_words(h, b)) * 4;
}

sf_status sf_project(sf_handle* h, void* stream, const sf_batch* b, int K, int form, const float* xi0,
                     const float* lam0, float* xi_out, float* lam_out, float* resid_out,
                     float* resid_hist, void* workspace, size_t workspace_bytes, void* checkpoints) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s0 = check_batch(h, b, &R, &S);
  if (s0 != SF_OK) return s0;
  if (K < 1) return fail(h, SF_ERR_INVALID_ARG, "K must be >= 1");
  if (S > 0 && (!xi_out || !lam_out || !resid_out))
    return fail(h, SF_ERR_INVALID_ARG, "xi_out / lambda_out / residual_out is NULL");
  if (form != SF_FORM_FUSED && form != SF_FORM_PLAIN) return fail(h, SF_ERR_INVALID_ARG, "unknown form");
  if (form == SF_FORM_PLAIN && h->pb.precision != SF_PREC_FP32)
    return fail(h, SF_ERR_UNSUPPORTED, "the plain form is float32 only");
  if (S == 0) return SF_OK;
  DeviceGuard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int dim = h->pb.dim, T = h->pb.T;
  const ProblemConsts pc = consts(h->pb, K);

  if (form == SF_FORM_PLAIN) {
    const size_t need = sf_workspace_bytes(h, b, form, K);
    if (!workspace || workspace_bytes < need)
      return fail(h, SF_ERR_WORKSPACE, "plain form needs " + std::to_string(need) + " workspace bytes");
    long long roff = 0, soff = 0, coff = 0;
    float* ws = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
    for (int sc = 0; sc < b->n_scenes; ++sc) {
      const int N = b->n_robots[sc], Ss = b->n_samples[sc];
      const size_t n = (size_t)Ss * dim * N * NV;
      const size_t xs = (size_t)Ss * 3 * dim * N * (size_t)T;
      PlainArgs a;
      a.pc = pc;
      a.basis = reinterpret_cast<const float4*>(h->basis);
      a.ops = h->ops;
      a.N = N;
      a.S = Ss;
      a.start = b->start + roff * dim;
      a.goal = b->goal + roff * dim;
      a.start_va = b->start_va ? b->start_va + roff * 2 * dim : nullptr;
      a.goal_va = b->goal_va ? b->goal_va + roff * 2 * dim : nullptr;
      a.xi_bar = b->xi_bar + coff;
      a.xi = xi_out + coff;
      a.lam = lam_out + coff;
      a.resid_out = resid_out + soff;
      a.hist = resid_hist ? resid_hist + soff : nullptr;
      a.hist_stride = (int)S;
      a.beta = ws;
      a.X = ws + (size_t)dim * N * NP;
      a.Q = a.X + xs;
      a.g = a.Q + xs;
      a.xprev = a.g + n;
      a.r2 = a.xprev + n;
      a.status = h->status;
      cudaError_t e = launch_plain(a, xi0 ? xi0 + coff : nullptr, lam0 ? lam0 + coff : nullptr, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "plain form launch");
      if (Ss > 0) h->launches += 2 + 4ULL * K + 3;
      roff += N;
      soff += Ss;
      coff += (long long)n;
    }
    return SF_OK;
  }

  FusedRequest rq;
  rq.xi0 = xi0;
  rq.lam0 = lam0;
  rq.xi_out = xi_out;
  rq.lam_out = lam_out;
  rq.resid_out = resid_out;
  rq.hist = resid_hist;
  rq.ckpt = reinterpret_cast<float*>(checkpoints);
  rq.prec = forward_form(h);
  if (checkpoints && h->pb.checkpoint_every <= 0)
    return fail(h, SF_ERR_INVALID_ARG, "checkpoints need a handle with checkpoint_every > 0");
  return run_fused(h, st, b, K, S, rq);
}

sf_status sf_project_train(sf_handle* h, void* stream, const sf_batch* b, int K, const float* xi0,
                           const float* lam0, float* xi_out, float* lam_out, float* resid_out, float* fp_res2_out,
                           void* checkpoints) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s0 = check_batch(h, b, &R, &S);
  if (s0 != SF_OK) return s0;
  if (K < 1) return fail(h, SF_ERR_INVALID_ARG, "K must be >= 1");
  if (h->pb.checkpoint_every <= 0) return fail(h, SF_ERR_INVALID_ARG, "handle has checkpoint_every = 0");
  if (S > 0 && (!xi_out || !lam_out || !resid_out || !checkpoints))
    return fail(h, SF_ERR_INVALID_ARG, "xi_out / lambda_out / residual_out / checkpoints is NULL");
  if (S == 0) return SF_OK;
  DeviceGuard g(h->device);
  FusedRequest rq;
  rq.xi0 = xi0;
  rq.lam0 = lam0;
  rq.xi_out = xi_out;
  rq.lam_out = lam_out;
  rq.resid_out = resid_out;
  rq.ckpt = reinterpret_cast<float*>(checkpoints);
  rq.fp_res2 = fp_res2_out;
  rq.prec = forward_form(h);
  return run_fused(h, reinterpret_cast<cudaStream_t>(stream), b, K, S, rq);
}

size_t sf_backward_workspace_bytes(const sf_handle* hc, const sf_batch* b, int K) {
  sf_handle* h = const_cast<sf_handle*>(hc);
  if (!h || h->pb.checkpoint_every <= 0 || K < 1) return 0;
  long long R = 0, S = 0;
  if (check_batch(h, b, &R, &S) != SF_OK) return 0;
  // ring of states, then the activity masks of the recomputed segment
  const long long ck = h->pb.checkpoint_every;
  return (size_t)(states_floats_aligned(ck + 1, total_coefs(h, b)) + ck * mask_slot_words(h, b)) * 4;
}

sf_status sf_project_backward(sf_handle* h, void* stream, const sf_batch* b, int K, int init_from_xi_bar,
                              const void* checkpoints, const float* g_xi, const float* g_lam, const float* g_fp,
                              float* gx0, float* gl0, float* gxb, void* workspace, size_t workspace_bytes) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s0 = check_batch(h, b, &R, &S);
  if (s0 != SF_OK) return s0;
  if (K < 1) return fail(h, SF_ERR_INVALID_ARG, "K must be >= 1");
  if (h->pb.checkpoint_every <= 0) return fail(h, SF_ERR_INVALID_ARG, "handle has checkpoint_every = 0");
  // the adjoint runs in float32 in every precision mode (its recompute of a
  // checkpoint segment is the float32 form's iteration)
  if (S == 0) return SF_OK;
  if (!checkpoints) return fail(h, SF_ERR_INVALID_ARG, "checkpoints is NULL");
  const size_t need = sf_backward_workspace_bytes(h, b, K);
  if (!workspace || workspace_bytes < need)
    return fail(h, SF_ERR_WORKSPACE, "backward needs " + std::to_string(need) + " workspace bytes");
  DeviceGuard g(h->device);
  FusedRequest rq;
  rq.backward = true;
  rq.bwd.ckpt = reinterpret_cast<const float*>(checkpoints);
  rq.bwd.ck_every = h->pb.checkpoint_every;
  rq.bwd.total_coefs = total_coefs(h, b);
  rq.bwd.ring = reinterpret_cast<float*>(workspace);
  {
    const long long ck = h->pb.checkpoint_every, nck = (K + ck - 1) / ck, tot = rq.bwd.total_coefs;
    rq.bwd.tail_mask = reinterpret_cast<const unsigned*>(rq.bwd.ckpt + states_floats_aligned(nck + ck + 1, tot));
    rq.bwd.ring_mask = reinterpret_cast<unsigned*>(rq.bwd.ring + states_floats_aligned(ck + 1, tot));
    rq.bwd.mask_slot = mask_slot_words(h, b);
  }
  rq.bwd.g_xi = g_xi;
  rq.bwd.g_lam = g_lam;
  rq.bwd.g_fp = g_fp;
  rq.bwd.gx0 = gx0;
  rq.bwd.gl0 = gl0;
  rq.bwd.gxb = gxb;
  rq.bwd.xi0_is_xi_bar = init_from_xi_bar ? 1 : 0;
  return run_fused(h, reinterpret_cast<cudaStream_t>(stream), b, K, S, rq);
}

namespace {
// Launches the QP layer over the batch's coefficient rows, at most
// MAX_SCENES_PER_LAUNCH scenes per launch (rows of consecutive scenes are
// contiguous, so each launch covers one contiguous row range).
sf_status run_eq(sf_handle* h, cudaStream_t st, const sf_batch* b, const float* in, float* out, float* grad_b,
                 bool backward) {
  const int dim = h->pb.dim;
  long long row = 0, roff = 0;
  int q = 0;
  while (q < b->n_scenes) {
    EqArgs a;
    std::memset(&a, 0, sizeof(a));
    a.start = b->start;
    a.goal = b->goal;
    a.start_va = b->start_va;
    a.goal_va = b->goal_va;
    std::memcpy(a.Pi, h->eq_pi, sizeof(a.Pi));
    std::memcpy(a.R, h->eq_r, sizeof(a.R));
    a.dim = dim;
    a.backward = backward ? 1 : 0;
    const long long first_row = row;
    int n = 0;
    for (; q < b->n_scenes && n < MAX_SCENES_PER_LAUNCH; ++q, ++n) {
      if ((long long)b->n_samples[q] * dim * b->n_robots[q] >= (1LL << 31))
        return fail(h, SF_ERR_INVALID_ARG, "a scene has 2^31 or more coefficient rows");
      a.sc[n].row_begin = row - first_row;
      a.sc[n].N = b->n_robots[q];
      a.sc[n].robot_off = (int)roff;
      row += (long long)b->n_samples[q] * dim * b->n_robots[q];
      roff += b->n_robots[q];
    }
    a.n_scenes = n;
    a.rows = row - first_row;
    a.in = in + first_row * NV;
    a.out = out + first_row * NV;
    a.grad_b = grad_b ? grad_b + first_row * 6 : nullptr;
    const cudaError_t e = launch_eq(a, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "QP layer launch");
    h->launches += a.rows > 0 ? 1 : 0;
  }
  return SF_OK;
}
}  // namespace

sf_status sf_eq_project(sf_handle* h, void* stream, const sf_batch* b, float* xi_out) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s0 = check_batch(h, b, &R, &S);
  if (s0 != SF_OK) return s0;
  if (S == 0) return SF_OK;
  if (!xi_out) return fail(h, SF_ERR_INVALID_ARG, "xi_out is NULL");
  DeviceGuard g(h->device);
  return run_eq(h, reinterpret_cast<cudaStream_t>(stream), b, b->xi_bar, xi_out, nullptr, false);
}

sf_status sf_eq_project_backward(sf_handle* h, void* stream, const sf_batch* b, const float* grad_out,
                                 float* grad_in, float* grad_b) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s0 = check_batch(h, b, &R, &S);
  if (s0 != SF_OK) return s0;
  if (S == 0) return SF_OK;
  if (!grad_out || !grad_in) return fail(h, SF_ERR_INVALID_ARG, "grad_out / grad_in is NULL");
  DeviceGuard g(h->device);
  return run_eq(h, reinterpret_cast<cudaStream_t>(stream), b, grad_out, grad_in, grad_b, true);
}

struct sf_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

sf_status sf_autotune(sf_handle* h, void* stream, const sf_batch* b, int K_probe, int n_candidates, float* xi_out,
                      float* lam_out, float* resid_out) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s0 = check_batch(h, b, &R, &S);
  if (s0 != SF_OK) return s0;
  if (K_probe < 1 || n_candidates < 1 || n_candidates > 64)
    return fail(h, SF_ERR_INVALID_ARG, "K_probe >= 1 and 1 <= n_candidates <= 64");
  if (S > 0 && (!xi_out || !lam_out || !resid_out)) return fail(h, SF_ERR_INVALID_ARG, "outputs are NULL");
  if (S == 0) return SF_OK;
  DeviceGuard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  FusedRequest rq;
  rq.xi_out = xi_out;
  rq.lam_out = lam_out;
  rq.resid_out = resid_out;
  rq.prec = forward_form(h);
  const int fG = h->force_G, fW = h->force_warps, fT = h->force_tc;
  h->force_G = h->force_warps = h->force_tc = 0;
  h->use_tuned = false;
  std::vector<LaunchGroup> gs;
  sf_status s = build_groups(h, b, K_probe, S, rq, &gs);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (size_t gi = 0; s == SF_OK && e == cudaSuccess && gi < gs.size(); ++gi) {
    LaunchGroup lg = gs[gi];
    std::vector<int> nr, ns;
    for (int q = 0; q < lg.a.n_scenes; ++q) {
      nr.push_back(lg.a.sc[q].N);
      ns.push_back(lg.a.sc[q].S);
    }
    std::vector<FusedPlan> top(n_candidates);
    plan_fused(h->pb.dim, lg.l.nmax, h->pb.T, nr.data(), ns.data(), (int)nr.size(), h->num_sms, h->max_smem_optin,
               0, 0, 0, false, top.data(), n_candidates, lg.l.prec);
    float best_ms = INFINITY;
    FusedPlan best = top[0];
    for (int c = 0; c < n_candidates && e == cudaSuccess; ++c) {
      const FusedPlan& p = top[c];
      if (p.G == 0) continue;
      LaunchGroup t = lg;
      int ctas = 0, gmax = 1;
      for (int q = 0; q < t.a.n_scenes; ++q) {
        SceneDesc& d = t.a.sc[q];
        d.G = std::min(p.G, d.S);
        d.cta_begin = ctas;
        ctas += (d.S + d.G - 1) / d.G;
        gmax = std::max(gmax, d.G);
      }
      t.a.tc = p.tc;
      t.a.nq = p.nq;
      t.l.n_ctas = ctas;
      t.l.gmax = gmax;
      t.l.warps = p.warps;
      t.l.tc = p.tc;
      t.l.nq = p.nq;
      t.l.smem = fused_smem_bytes(h->pb.dim, t.l.nmax, h->pb.T, gmax, p.tc, p.nq, false, t.l.prec);
      if (t.l.smem > h->max_smem_optin) continue;
      float ms_sum = 0.0f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // first run warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_group(t, rq, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_sum += ms;
        h->launches += 1;
      }
      if (e == cudaSuccess && ms_sum < best_ms) {
        best_ms = ms_sum;
        best = p;
      }
    }
    if (e == cudaSuccess) h->tuned[lg.key] = best;   // the key does not depend on K
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->force_G = fG;
  h->force_warps = fW;
  h->force_tc = fT;
  h->use_tuned = true;
  if (s != SF_OK) return s;
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  return SF_OK;
}

sf_status sf_graph_capture(sf_handle* h, const sf_batch* b, int K, int form, const float* xi0, const float* lam0,
                           float* xi_out, float* lam_out, float* resid_out, float* resid_hist, void* workspace,
                           size_t workspace_bytes, sf_graph** out) {
  if (!h || !out) return SF_ERR_INVALID_ARG;
  *out = nullptr;
  DeviceGuard g(h->device);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(h, e, "capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(h, e, "begin capture");
  }
  sf_status s = sf_project(h, cs, b, K, form, xi0, lam0, xi_out, lam_out, resid_out, resid_hist, workspace,
                           workspace_bytes, nullptr);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (s != SF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  sf_graph* gr = new (std::nothrow) sf_graph();
  if (!gr) {
    cudaGraphDestroy(graph);
    return SF_ERR_OOM;
  }
  gr->graph = graph;
  gr->device = h->device;
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    delete gr;
    return cuda_fail(h, e, "graph instantiate");
  }
  *out = gr;
  return SF_OK;
}

sf_status sf_graph_launch(sf_graph* gr, void* stream) {
  if (!gr) return SF_ERR_INVALID_ARG;
  DeviceGuard g(gr->device);
  return cudaGraphLaunch(gr->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

void sf_graph_destroy(sf_graph* gr) {
  if (!gr) return;
  DeviceGuard g(gr->device);
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  delete gr;
}

unsigned long long sf_launch_count(const sf_handle* h) { return h ? h->launches : 0ULL; }

sf_status sf_set_launch_shape(sf_handle* h, int G, int warps, int tc) {
  if (!h) return SF_ERR_INVALID_ARG;
  if (G > 64 || warps > 32 || tc > SF_MAX_T) return fail(h, SF_ERR_INVALID_ARG, "launch shape out of range");
  h->force_G = G > 0 ? G : 0;
  h->force_warps = warps > 0 ? warps : 0;
  h->force_tc = tc > 0 ? tc : 0;
  return SF_OK;
}

sf_status sf_get_launch_shape(const sf_handle* h, int* out4) {
  if (!h || !out4) return SF_ERR_INVALID_ARG;
  for (int q = 0; q < 4; ++q) out4[q] = h->last_plan[q];
  return SF_OK;
}

sf_status sf_get_launch_form(const sf_handle* h, int* tensor_memory) {
  if (!h || !tensor_memory) return SF_ERR_INVALID_ARG;
  *tensor_memory = h->last_form;
  return SF_OK;
}

namespace {
struct HostPlan {
  size_t off_start, off_goal, off_sva, off_gva, off_xib, off_xi0, off_lam0, off_xi, off_lam, off_res,
      off_ws, total;
  long long R, S, coefs;
  size_t ws;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

sf_status host_plan(sf_handle* h, const sf_batch* b, int form, int K, HostPlan* p) {
  sf_status s = check_batch(h, b, &p->R, &p->S);
  if (s != SF_OK) return s;
  if (K < 1) return fail(h, SF_ERR_INVALID_ARG, "K must be >= 1");
  const int dim = h->pb.dim;
  p->coefs = 0;
  for (int sc = 0; sc < b->n_scenes; ++sc) p->coefs += (long long)b->n_samples[sc] * dim * b->n_robots[sc] * NV;
  p->ws = sf_workspace_bytes(h, b, form, K);
  size_t o = 0;
  const size_t pos = sizeof(float) * (size_t)p->R * dim, va = 2 * pos, cf = sizeof(float) * (size_t)p->coefs;
  p->off_start = o; o = align256(o + pos);
  p->off_goal = o; o = align256(o + pos);
  p->off_sva = o; o = align256(o + va);
  p->off_gva = o; o = align256(o + va);
  p->off_xib = o; o = align256(o + cf);
  p->off_xi0 = o; o = align256(o + cf);
  p->off_lam0 = o; o = align256(o + cf);
  p->off_xi = o; o = align256(o + cf);
  p->off_lam = o; o = align256(o + cf);
  p->off_res = o; o = align256(o + sizeof(float) * (size_t)p->S);
  p->off_ws = o; o = align256(o + p->ws);
  p->total = o + 256;
  return SF_OK;
}
}  // namespace

size_t sf_host_staging_bytes(const sf_handle* hc, const sf_batch* b, int form, int K) {
  sf_handle* h = const_cast<sf_handle*>(hc);
  if (!h) return 0;
  HostPlan p;
  if (host_plan(h, b, form, K, &p) != SF_OK) return 0;
  return p.total;
}

sf_status sf_project_host(sf_handle* h, void* stream, const sf_batch* b, int K, int form, const float* xi0,
                          const float* lam0, float* xi_out, float* lam_out, float* resid_out,
                          void* staging, size_t staging_bytes) {
  if (!h) return SF_ERR_INVALID_ARG;
  HostPlan p;
  sf_status s = host_plan(h, b, form, K, &p);
  if (s != SF_OK) return s;
  if (p.S > 0 && (!xi_out || !lam_out || !resid_out))
    return fail(h, SF_ERR_INVALID_ARG, "xi_out / lambda_out / residual_out is NULL");
  if (!staging || staging_bytes < p.total)
    return fail(h, SF_ERR_WORKSPACE, "staging needs " + std::to_string(p.total) + " bytes");
  DeviceGuard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(staging) + 255) & ~uintptr_t(255));
  const int dim = h->pb.dim;
  const size_t pos = sizeof(float) * (size_t)p.R * dim, cf = sizeof(float) * (size_t)p.coefs;
  auto h2d = [&](size_t off, const void* src, size_t n) -> cudaError_t {
    return (src && n) ? cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  cudaError_t e = h2d(p.off_start, b->start, pos);
  if (e == cudaSuccess) e = h2d(p.off_goal, b->goal, pos);
  if (e == cudaSuccess) e = h2d(p.off_sva, b->start_va, 2 * pos);
  if (e == cudaSuccess) e = h2d(p.off_gva, b->goal_va, 2 * pos);
  if (e == cudaSuccess) e = h2d(p.off_xib, b->xi_bar, cf);
  if (e == cudaSuccess) e = h2d(p.off_xi0, xi0, cf);
  if (e == cudaSuccess) e = h2d(p.off_lam0, lam0, cf);
  if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
  sf_batch db = *b;
  db.start = reinterpret_cast<const float*>(base + p.off_start);
  db.goal = reinterpret_cast<const float*>(base + p.off_goal);
  db.start_va = b->start_va ? reinterpret_cast<const float*>(base + p.off_sva) : nullptr;
  db.goal_va = b->goal_va ? reinterpret_cast<const float*>(base + p.off_gva) : nullptr;
  db.xi_bar = reinterpret_cast<const float*>(base + p.off_xib);
  float* dxi = reinterpret_cast<float*>(base + p.off_xi);
  float* dlam = reinterpret_cast<float*>(base + p.off_lam);
  float* dres = reinterpret_cast<float*>(base + p.off_res);
  s = sf_project(h, stream, &db, K, form, xi0 ? reinterpret_cast<const float*>(base + p.off_xi0) : nullptr,
                 lam0 ? reinterpret_cast<const float*>(base + p.off_lam0) : nullptr, dxi, dlam, dres, nullptr,
                 p.ws ? base + p.off_ws : nullptr, p.ws, nullptr);
  if (s != SF_OK) return s;
  e = cudaMemcpyAsync(xi_out, dxi, cf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lam_out, dlam, cf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(resid_out, dres, sizeof(float) * (size_t)p.S, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
  return SF_OK;
}

// ---- plain form on a built-in scratch buffer (no device allocation) -------
//
// For callers that may not allocate device memory when they call in: the
// time-domain arrays of the plain form live in this static device array
// instead of a caller-provided workspace. In host code the name below is a
// host-side stand-in, not a device address; the device address is looked up
// once per device with cudaGetSymbolAddress and then passed to the kernels.
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[SF_NOALLOC_SCRATCH_BYTES];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoallocSlot {
  void* addr;                 // device address of the buffer
  unsigned long long ctx_id;  // id of the context it was looked up in (0: unknown)
};
NoallocSlot g_noalloc[kMaxDevices] = {};

// Id of the calling thread's current context, unique for the life of the
// process (a context created after cudaDeviceReset gets a new one); 0 when
// the driver does not provide it. The driver calls are reached through the
// runtime's entry-point table, so the library needs no link to libcuda.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {   // under g_noalloc_mu
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the buffer on h->device (the caller has made that device
// current and the runtime has initialised its context). Looked up on the
// first call per device, and again whenever the current context is not the
// one of the last lookup (after cudaDeviceReset the old address is stale).
sf_status noalloc_scratch_address(sf_handle* h, void** out) {
  if (h->device < 0 || h->device >= kMaxDevices) return fail(h, SF_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocSlot& slot = g_noalloc[h->device];
  const unsigned long long ctx = current_context_id();
  if (!slot.addr || ctx == 0 || ctx != slot.ctx_id) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(h, e, "device address of the built-in scratch buffer");
    slot.addr = p;
    slot.ctx_id = ctx;
  }
  *out = slot.addr;
  return SF_OK;
}
}  // namespace

sf_status sf_project_plain_noalloc(sf_handle* h, void* stream, const sf_batch* b, int K, const float* xi0,
                                   const float* lam0, float* xi_out, float* lam_out, float* resid_out,
                                   float* resid_hist) {
  if (!h) return SF_ERR_INVALID_ARG;
  long long R = 0, S = 0;
  sf_status s = check_batch(h, b, &R, &S);
  if (s != SF_OK) return s;
  if (K < 1) return fail(h, SF_ERR_INVALID_ARG, "K must be >= 1");
  const size_t need = sf_workspace_bytes(h, b, SF_FORM_PLAIN, K);
  if (need > (size_t)SF_NOALLOC_SCRATCH_BYTES)
    return fail(h, SF_ERR_INVALID_ARG,
                "batch needs " + std::to_string(need) + " bytes of plain-form scratch; the built-in buffer of "
                "sf_project_plain_noalloc holds " + std::to_string((size_t)SF_NOALLOC_SCRATCH_BYTES) +
                " bytes (split the batch into smaller scenes or sample ranges)");
  DeviceGuard g(h->device);
  void* scratch = nullptr;
  s = noalloc_scratch_address(h, &scratch);
  if (s != SF_OK) return s;
  return sf_project(h, stream, b, K, SF_FORM_PLAIN, xi0, lam0, xi_out, lam_out, resid_out, resid_hist, scratch,
                    (size_t)SF_NOALLOC_SCRATCH_BYTES, nullptr);
}

sf_status sf_plan_launch(int dim, int T, int n_scenes, const int* n_robots, const int* n_samples, int precision,
                         int num_sms, size_t smem_per_block_optin, int* out4, size_t* out_smem) {
  if ((dim != 2 && dim != 3) || T < 2 || T > SF_MAX_T || n_scenes < 1 || n_scenes > MAX_SCENES_PER_LAUNCH ||
      !n_robots || !n_samples || !out4 || num_sms < 1 || precision < SF_PREC_FP32 || precision > SF_PREC_FP16)
    return SF_ERR_INVALID_ARG;
  int bk = -1;
  long long total = 0;
  for (int q = 0; q < n_scenes; ++q) {
    if (n_robots[q] < 1 || n_robots[q] > SF_MAX_ROBOTS || n_samples[q] < 0) return SF_ERR_INVALID_ARG;
    const int b = bucket_index(n_robots[q]);
    if (bk >= 0 && b != bk) return SF_ERR_INVALID_ARG;   // one robot-count bucket per launch group
    bk = b;
    total += n_samples[q];
  }
  if (total < 1) return SF_ERR_INVALID_ARG;
  // the form a handle of this precision uses by default (16-bit: tensor memory)
  const int form = precision == SF_PREC_FP32 ? 0 : PREC_TM_TF32 + precision;
  const FusedPlan p = plan_fused(dim, kBucketNmax[bk], T, n_robots, n_samples, n_scenes, num_sms,
                                 smem_per_block_optin, 0, 0, 0, false, nullptr, 0, form);
  if (p.G == 0) return SF_ERR_UNSUPPORTED;
  out4[0] = p.G;
  out4[1] = p.warps;
  out4[2] = p.tc;
  out4[3] = p.nq;
  if (out_smem) *out_smem = p.smem;
  return SF_OK;
}

sf_status sf_set_option(sf_handle* h, int option, int value) {
  if (!h) return SF_ERR_INVALID_ARG;
  if (option == SF_OPT_PAIR_PRUNING) {
    if (value != 0 && value != 1) return fail(h, SF_ERR_INVALID_ARG, "SF_OPT_PAIR_PRUNING takes 0 or 1");
    h->prune = value;
    return SF_OK;
  }
  if (option == SF_OPT_TENSOR_MEMORY) {
    if (value < 0 || value > 2) return fail(h, SF_ERR_INVALID_ARG, "SF_OPT_TENSOR_MEMORY takes 0, 1 or 2");
    h->tm = value;
    return SF_OK;
  }
  if (option == SF_OPT_TEST_WAIT_TIMEOUT) {
    if (value < 0 || value > 1000000)
      return fail(h, SF_ERR_INVALID_ARG, "SF_OPT_TEST_WAIT_TIMEOUT takes 0 .. 1000000 microseconds");
    h->wait_test_us = value;
    return SF_OK;
  }
  if (option == SF_OPT_TEST_CANARY) {
#if SF_DEBUG_CHECKS
    if (value != 0 && value != 1) return fail(h, SF_ERR_INVALID_ARG, "SF_OPT_TEST_CANARY takes 0 or 1");
    h->plant_canary = value;
    return SF_OK;
#else
    return fail(h, SF_ERR_UNSUPPORTED, "SF_OPT_TEST_CANARY needs a library built with SF_DEBUG_CHECKS");
#endif
  }
  return fail(h, SF_ERR_INVALID_ARG, "unknown option");
}

sf_status sf_sync_status(sf_handle* h, void* stream) {
  if (!h) return SF_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
  int word = 0;
  e = cudaMemcpy(&word, h->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  if (word) {
    cudaMemset(h->status, 0, sizeof(int));
    if (word & ST_TIMEOUT) return fail(h, SF_ERR_TIMEOUT, "a bounded device wait ran out");
    if (word & ST_DEBUG)
      return fail(h, SF_ERR_DEBUG_CHECK,
                  "debug check failed at site " + std::to_string((word >> 8) & 0xFF) + " (" +
                      debug_site_name((word >> 8) & 0xFF) + ")");
    if (word & ST_NONFINITE) return fail(h, SF_ERR_NONFINITE, "non-finite value in the output");
  }
  return SF_OK;
}

}  // extern "C"
