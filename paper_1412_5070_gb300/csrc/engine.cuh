// engine.cuh -- batched execution of requests (f12int_submit / f12int_poll).
//
// Included by f12int.cu after the kernels and the context definition.
//
// A request asks for the blocks of some classes over one quartet list of one
// basis.  A worker thread merges the pending requests -- of any bases and any
// mix of (la, lb, lc, ld) -- into a batch, writes the batch's lists to pinned
// staging memory, copies them to fixed device buffers and replays one
// captured CUDA graph.  The graph holds, for every class, the four passes of
// the auxiliary stage and one contraction launch per shared-memory tier, all
// persistent (grid-stride over counts read from device memory), so the same
// graph serves every batch.  The six class pipelines are parallel branches
// of the graph, each with its own work-item buffers.  Two staging buffers let the host build batch
// k+1 while batch k runs.  The method is that of f12int_compute_class; only
// the scheduling differs.

namespace {

constexpr int kTiers = 5;                // shared-memory tiers per precision
constexpr size_t kTierCap[kTiers] = {32 * 1024, 64 * 1024, 112 * 1024, 200 * 1024, 200 * 1024};
constexpr int kTierWarps[kTiers] = {4, 4, 4, 4, 2};   // the last for quartets that need fewer warps
constexpr int kLaunches = 2 * kTiers;     // FP64 tiers, then FP32 tiers (mixed requests)
constexpr int kThinSlot = kLaunches;      // then the thin contraction (total order <= 3, I5 <= 2), one
constexpr int kSlots = kLaunches + kThinKeys;   // launch per (la, lb, lc, ld)

struct EngineReq {
  uint64_t ticket = 0;
  int basis = 0;
  const f12int_ctx::BasisData *B = nullptr;   // stable: the deque never moves its elements
  uint32_t mask = 0;
  int precision = 0;                  // 1: FP32 recursion and contraction below the FP32 bound
  double thresh = 0.0;
  double *out = nullptr;
  std::vector<int32_t> q;
  std::vector<int64_t> off;       // [nclass][n]
  int64_t quartets[7] = {0};      // quartets per class (before screening)
  int64_t items[7] = {0};         // work items per class (before screening)
  int64_t tasks[7] = {0};         // contraction tasks per class (before screening)
};

struct TicketState {
  bool done = false;
  int rc = F12INT_OK;
  int batch = -1;                 // staging buffer of the batch that runs it
};

// Contraction plan of a quartet of nprimq primitive quartets in a batch:
// ket ranges at 4 warps (the fewest that fit the largest tier, more while a
// task would exceed kTaskFlops), the tier that holds them, and the work of
// one task.
struct BatchPlan {
  int tier, nsplit;
  double work;
};

static bool batch_plan(int la, int lb, int lc, int ld, int cls, int64_t nprimq, double target, BatchPlan *bp,
                       bool fp32 = false) {
  const int ncd = ncart(lc) * ncart(ld);
  if (thin_quartet((la << 6) | (lb << 4) | (lc << 2) | ld, cls)) {   // one warp, FP64 (mixed requests too)
    bp->tier = kThinSlot + thin_slot((la << 6) | (lb << 4) | (lc << 2) | ld, cls == 5);
    bp->nsplit = 1;
    bp->work = (double)nprimq * task_flops(la, lb, lc, ld, cls, ncd);
    return true;
  }
  const size_t esz = fp32 ? 4 : 8;
  // 4-warp tiers first; the 2-warp tier only for what no 4-warp tier holds
  for (int pass = 0; pass < 2; ++pass) {
    const int nw = pass == 0 ? 4 : 2;
    for (int ns = 1; ns <= ncd; ++ns) {
      if (!valid_split(ncd, ns)) continue;
      if (contract_smem(la, lb, lc, ld, cls, nw, ns, esz) > kTierCap[kTiers - 1]) continue;
      const int nsw = work_split(la, lb, lc, ld, cls, nprimq, ns, target);
      const size_t sm = contract_smem(la, lb, lc, ld, cls, nw, nsw, esz);
      for (int t = 0; t < kTiers; ++t)
        if (kTierWarps[t] == nw && sm <= kTierCap[t]) {
          bp->tier = t + (fp32 ? kTiers : 0);
          bp->nsplit = nsw;
          bp->work = (double)nprimq * task_flops(la, lb, lc, ld, cls, (ncd + nsw - 1) / nsw);
          return true;
        }
    }
  }
  return false;
}

// Per-class lists of a batch; the same layout on the device and in each
// pinned staging buffer.
struct ClassLists {
  int32_t *quartets = nullptr;    // [qcap][4]
  int64_t *pq_off = nullptr;      // [qcap + 1]
  int64_t *offsets = nullptr;     // [qcap]
  int32_t *qslot = nullptr;       // [qcap]
  CTask *tasks = nullptr;         // [tcap], tier after tier
  int64_t *counts = nullptr;      // n, npq, then (begin, end) of the tasks of each tier
  PairView *views = nullptr;      // [scap]
  double **outs = nullptr;        // [scap]
};
constexpr int kCounts = 2 + 2 * kSlots;

struct Engine {
  // limits
  int64_t qcap = (int64_t)1 << 19;   // quartets per class per batch
  int64_t icap = 0;                   // work items per class per batch (0: from free HBM)
  int64_t tcap = 0;                   // contraction tasks per class per batch
  int64_t scap = 4096;                // requests per batch
  int64_t zcap = 0;                   // zero-filled blocks per batch
  bool ready = false;
  // device buffers
  ClassLists dev[7];
  double **zero_dst = nullptr;
  int64_t *zero_len = nullptr, *zero_count = nullptr;
  int *keys[7] = {nullptr};             // per class: item keys, key order, histogram, partials
  unsigned *order[7] = {nullptr}, *hist[7] = {nullptr};
  double *part[7] = {nullptr};
  unsigned *status = nullptr;
  size_t bytes = 0;
  // staging (pinned), two buffers
  ClassLists stage[2][7];
  double **zstage_dst[2] = {nullptr, nullptr};
  int64_t *zstage_len[2] = {nullptr, nullptr}, *zstage_count[2] = {nullptr, nullptr};
  unsigned *stage_status[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<uint64_t> inflight[2];
  // graph
  cudaStream_t stream = nullptr;
  cudaStream_t branch[7] = {nullptr};   // capture streams of the class branches
  cudaGraphExec_t exec = nullptr;
  bool graph_dirty = true;
  int items_blocks = 0, quad_blocks = 0, classify_blocks = 0, tier_blocks[kLaunches] = {0};
  int thin_blocks = 0;           // persistent thin contraction launches
  double fp32_below = 1e-5;           // mixed requests: FP32 below this screening estimate
  // per-class schedule (f12int_batch_autotune): work target of a contraction
  // task and the divisor of the auxiliary-stage grid
  double task_target[7] = {kTaskFlops, kTaskFlops, kTaskFlops, kTaskFlops, kTaskFlops, kTaskFlops, kTaskFlops};
  int items_div[7] = {1, 1, 1, 1, 1, 1, 1};
  // queue
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<EngineReq *> pending;
  std::unordered_map<uint64_t, TicketState> tickets;
  uint64_t next_ticket = 1;
  int cur = 0;
  int64_t batches = 0, requests_done = 0;
};

template <class T>
static int engine_alloc(f12int_ctx *ctx, Engine &E, T **p, size_t n) {
  int rc = dalloc(ctx, p, sizeof(T) * std::max<size_t>(n, 1));
  if (rc == F12INT_OK) E.bytes += sizeof(T) * std::max<size_t>(n, 1);
  return rc;
}

template <class T>
static int stage_alloc(T **p, size_t n) {
  return cudaHostAlloc((void **)p, sizeof(T) * std::max<size_t>(n, 1), cudaHostAllocDefault) == cudaSuccess
             ? F12INT_OK
             : F12INT_ENOMEM;
}

static int lists_alloc_dev(f12int_ctx *ctx, Engine &E, ClassLists &L) {
  int rc = engine_alloc(ctx, E, &L.quartets, 4 * (size_t)E.qcap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.pq_off, (size_t)E.qcap + 1);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.offsets, (size_t)E.qcap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.qslot, (size_t)E.qcap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.tasks, (size_t)E.tcap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.counts, (size_t)kCounts);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.views, (size_t)E.scap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &L.outs, (size_t)E.scap);
  return rc;
}

static int lists_alloc_host(Engine &E, ClassLists &L) {
  int rc = stage_alloc(&L.quartets, 4 * (size_t)E.qcap);
  if (rc == F12INT_OK) rc = stage_alloc(&L.pq_off, (size_t)E.qcap + 1);
  if (rc == F12INT_OK) rc = stage_alloc(&L.offsets, (size_t)E.qcap);
  if (rc == F12INT_OK) rc = stage_alloc(&L.qslot, (size_t)E.qcap);
  if (rc == F12INT_OK) rc = stage_alloc(&L.tasks, (size_t)E.tcap);
  if (rc == F12INT_OK) rc = stage_alloc(&L.counts, (size_t)kCounts);
  if (rc == F12INT_OK) rc = stage_alloc(&L.views, (size_t)E.scap);
  if (rc == F12INT_OK) rc = stage_alloc(&L.outs, (size_t)E.scap);
  return rc;
}

static void lists_free(ClassLists &L, bool host) {
  void *ps[] = {L.quartets, L.pq_off, L.offsets, L.qslot, L.tasks, L.counts, L.views, L.outs};
  for (void *p : ps)
    if (p) host ? cudaFreeHost(p) : cudaFree(p);
  L = ClassLists{};
}

// Zero-fill the blocks of screened-out quartets.
__global__ void k_zero_blocks(double *const *dst, const int64_t *len, const int64_t *count) {
  const int64_t n = *count;
  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    double *d = dst[b];
    for (int64_t i = threadIdx.x; i < len[b]; i += blockDim.x) d[i] = 0.0;
  }
}

// Capture the launch sequence of one batch (every class, every tier).
static int engine_capture(f12int_ctx *ctx, Engine &E) {
  if (E.exec) {
    cudaGraphExecDestroy(E.exec);
    E.exec = nullptr;
  }
  for (int t = 0; t < kTiers; ++t)
    if (kTierCap[t] > 48 * 1024) {
      CK(cudaFuncSetAttribute(k_contract<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTierCap[t]));
      CK(cudaFuncSetAttribute(k_contract<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTierCap[t]));
    }
  cudaStream_t cs = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t fork = nullptr, join[7] = {nullptr};
  CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (int c = 1; c <= 6; ++c) CK(cudaEventCreateWithFlags(&join[c], cudaEventDisableTiming));
  const PairView none{};
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    k_zero_blocks<<<4 * 152, 128, 0, cs>>>(E.zero_dst, E.zero_len, E.zero_count);
    cudaEventRecord(fork, cs);
    for (int cls = 1; cls <= 6; ++cls) {
      cudaStream_t bs = E.branch[cls];
      cudaStreamWaitEvent(bs, fork, 0);
      const int kcls = cls == 5 ? 3 : cls;
      const int nf = ctx->tables.nfam[kcls];
      const ClassLists &L = E.dev[cls];
      QuartetView QV{L.quartets, L.pq_off, 0, L.counts, L.qslot, L.views, L.outs};
      cudaMemsetAsync(E.hist[cls], 0, sizeof(unsigned) * kNKeys, bs);
      k_items_classify<true><<<E.classify_blocks, BLOCK_AUX, 0, bs>>>(ctx->tables, none, QV, cls, 0, 0,
                                                                      E.keys[cls], E.hist[cls]);
      k_items_scan<<<1, 1024, 0, bs>>>(E.hist[cls], kNKeys);
      k_items_scatter<<<E.classify_blocks, BLOCK_AUX, 0, bs>>>(QV, nf, 0, E.keys[cls], E.hist[cls], 0,
                                                               E.order[cls]);
      k_items_eval<true><<<std::max(1, E.items_blocks / E.items_div[cls]), BLOCK_AUX, 0, bs>>>(
          ctx->tables, none, QV, cls, 0, 0, E.order[cls], E.keys[cls],
                                                               E.part[cls], E.status, nullptr);
      if (ctx->cls_quad[cls])   // families evaluated by quadrature (b < 0, alpha0 < -1)
        k_items_eval<true, true><<<E.quad_blocks, BLOCK_AUX, 0, bs>>>(ctx->tables, none, QV, cls, 0, 0,
                                                                       E.order[cls], E.keys[cls], E.part[cls],
                                                                       E.status, nullptr);
      for (int t = 0; t < kLaunches; ++t) {
        const int tt = t % kTiers;
        if (t < kTiers)
          k_contract<true, double><<<E.tier_blocks[t], 32 * kTierWarps[tt], kTierCap[tt], bs>>>(
              none, QV, cls, nf, 0, L.tasks, 0, L.counts + 2 + 2 * t, E.keys[cls], E.part[cls], nullptr, L.offsets,
              E.status, nullptr);
        else
          k_contract<true, float><<<E.tier_blocks[t], 32 * kTierWarps[tt], kTierCap[tt], bs>>>(
              none, QV, cls, nf, 0, L.tasks, 0, L.counts + 2 + 2 * t, E.keys[cls], E.part[cls], nullptr, L.offsets,
              E.status, nullptr);
      }
      // one persistent launch per thin (la, lb, lc, ld) of the class kind
      for (int k = 0; k < 256; ++k) {
        const int slot = thin_quartet(k, cls) ? thin_slot(k, cls == 5) : -1;
        if (slot < 0) continue;
        thin_kernel(k, cls == 5)<<<E.thin_blocks, 32 * kThinWarps, 0, bs>>>(
            none, QV, nf, 0, L.tasks, 0, L.counts + 2 + 2 * (kThinSlot + slot), E.keys[cls], E.part[cls], nullptr,
            L.offsets, nullptr);
      }
      cudaEventRecord(join[cls], bs);
      cudaStreamWaitEvent(cs, join[cls], 0);
    }
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&E.exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaEventDestroy(fork);
  for (int c = 1; c <= 6; ++c) cudaEventDestroy(join[c]);
  if (e != cudaSuccess) return cuda_fail(e);
  E.graph_dirty = false;
  return F12INT_OK;
}

// Buffers, streams and launch shapes; called once, at the first submit.
static int engine_init(f12int_ctx *ctx, Engine &E) {
  if (E.icap == 0) {
    // admission by free device memory: the six classes' item buffers take at
    // most a quarter of what is free (and of what the budget leaves)
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    if (ctx->budget) free_b = std::min(free_b, ctx->budget > ctx->used ? ctx->budget - ctx->used : (size_t)0);
    const size_t per_item = sizeof(int) + sizeof(unsigned) + sizeof(double) * kPartPitch;
    const int64_t fit = (int64_t)(free_b / 4 / (6 * per_item));
    E.icap = std::min<int64_t>((int64_t)1 << 26, fit);
    if (E.icap < ((int64_t)1 << 16)) return F12INT_ENOMEM;
  }
  E.tcap = 4 * E.qcap;
  E.zcap = 6 * E.qcap;
  int rc = F12INT_OK;
  for (int c = 1; c <= 6 && rc == F12INT_OK; ++c) rc = lists_alloc_dev(ctx, E, E.dev[c]);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.zero_dst, (size_t)E.zcap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.zero_len, (size_t)E.zcap);
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.zero_count, 1);
  for (int c = 1; c <= 6 && rc == F12INT_OK; ++c) {
    rc = engine_alloc(ctx, E, &E.keys[c], (size_t)E.icap);
    if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.order[c], (size_t)E.icap);
    if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.part[c], (size_t)E.icap * kPartPitch);
    if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.hist[c], (size_t)kNKeys);
    if (rc == F12INT_OK && cudaStreamCreateWithFlags(&E.branch[c], cudaStreamNonBlocking) != cudaSuccess)
      rc = F12INT_ECUDA;
  }
  if (rc == F12INT_OK) rc = engine_alloc(ctx, E, &E.status, 1);
  for (int b = 0; b < 2 && rc == F12INT_OK; ++b) {
    for (int c = 1; c <= 6 && rc == F12INT_OK; ++c) rc = lists_alloc_host(E, E.stage[b][c]);
    if (rc == F12INT_OK) rc = stage_alloc(&E.zstage_dst[b], (size_t)E.zcap);
    if (rc == F12INT_OK) rc = stage_alloc(&E.zstage_len[b], (size_t)E.zcap);
    if (rc == F12INT_OK) rc = stage_alloc(&E.zstage_count[b], 1);
    if (rc == F12INT_OK) rc = stage_alloc(&E.stage_status[b], 1);
    if (rc == F12INT_OK && cudaEventCreateWithFlags(&E.ev[b], cudaEventDisableTiming) != cudaSuccess)
      rc = F12INT_ECUDA;
  }
  if (rc == F12INT_OK && cudaStreamCreateWithFlags(&E.stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = F12INT_ECUDA;
  if (rc == F12INT_OK && cudaMemset(E.status, 0, sizeof(unsigned)) != cudaSuccess) rc = F12INT_ECUDA;
  if (rc != F12INT_OK) return rc;
  // persistent launch shapes: resident blocks per SM from registers and shared memory
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  int per = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_items_eval<true>, BLOCK_AUX, 0));
  E.items_blocks = nsm * std::max(per, 1);
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_items_eval<true, true>, BLOCK_AUX, 0));
  E.quad_blocks = nsm * std::max(per, 1);
  E.classify_blocks = nsm * 8;
  for (int t = 0; t < kTiers; ++t) {
    if (kTierCap[t] > 48 * 1024) {
      CK(cudaFuncSetAttribute(k_contract<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTierCap[t]));
      CK(cudaFuncSetAttribute(k_contract<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTierCap[t]));
    }
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_contract<true, double>, 32 * kTierWarps[t],
                                                     kTierCap[t]));
    E.tier_blocks[t] = nsm * std::max(per, 1);
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_contract<true, float>, 32 * kTierWarps[t],
                                                     kTierCap[t]));
    E.tier_blocks[kTiers + t] = nsm * std::max(per, 1);
  }
  E.thin_blocks = nsm * 4;   // 16 warps per SM: the thin launches of a batch are mostly small
  E.ready = true;
  return F12INT_OK;
}

// Mark the requests of the batch in staging buffer b done (the batch's event
// has completed).  Caller holds E.mu.
static void engine_finish_batch(Engine &E, int b) {
  const int rc = *E.stage_status[b] ? F12INT_EDEVICE : F12INT_OK;
  for (uint64_t t : E.inflight[b]) {
    auto it = E.tickets.find(t);
    if (it != E.tickets.end()) {
      it->second.done = true;
      it->second.rc = rc;
      it->second.batch = -1;
    }
    ++E.requests_done;
  }
  E.inflight[b].clear();
}

// Build the lists of one batch in staging buffer b and launch it.
static int engine_launch(f12int_ctx *ctx, Engine &E, const std::vector<EngineReq *> &batch, int b) {
  struct Item {
    int64_t src;      // index into the flat per-class arrays below
    int tier, nsplit;
    double work;      // per task
  };
  int64_t nzero = 0;
  for (int cls = 1; cls <= 6; ++cls) {
    ClassLists &S = E.stage[b][cls];
    int64_t n = 0;
    std::vector<Item> items;
    // gather the class's quartets of every request
    for (size_t r = 0; r < batch.size(); ++r) {
      const EngineReq &R = *batch[r];
      if (!(R.mask & (1u << (cls - 1)))) continue;
      int row = 0;
      for (int c = 1; c < cls; ++c) row += (R.mask >> (c - 1)) & 1;
      const f12int_ctx::BasisData &B = *R.B;
      const int nq = (int)(R.q.size() / 4);
      const bool mixed = R.precision == 1;
      for (int i = 0; i < nq; ++i) {
        const int32_t *s = &R.q[4 * (size_t)i];
        const int64_t off = R.off[(size_t)row * nq + i];
        const int la = B.l[s[0]], lb = B.l[s[1]], lc = B.l[s[2]], ld = B.l[s[3]];
        const double est =
            (R.thresh > 0.0 || mixed) ? screen_estimate(ctx, B, cls, s[0], s[1], s[2], s[3]) : 0.0;
        if (R.thresh > 0.0 && est < R.thresh) {
          E.zstage_dst[b][nzero] = R.out + off;
          E.zstage_len[b][nzero] = (int64_t)ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
          ++nzero;
          continue;
        }
        BatchPlan bp{};
        const int64_t np = (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]];
        const bool fp32 = mixed && est < E.fp32_below;
        batch_plan(la, lb, lc, ld, cls, np, E.task_target[cls], &bp, fp32);   // checked at submit
        for (int k = 0; k < 4; ++k) S.quartets[4 * n + k] = s[k];
        S.offsets[n] = off;
        S.qslot[n] = (int32_t)r;
        items.push_back(Item{n, bp.tier, bp.nsplit, bp.work});
        ++n;
      }
      S.views[r] = pair_view(ctx, B, cls, B.prim_screen);
      S.outs[r] = R.out;
    }
    // working order: by tier, then decreasing work per task (the longest
    // tasks start first); permute the lists
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) {
      if (x.tier != y.tier) return x.tier < y.tier;
      return x.work > y.work;
    });
    std::vector<int32_t> q2((size_t)4 * n), sl2((size_t)n);
    std::vector<int64_t> of2((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t j = items[i].src;
      for (int k = 0; k < 4; ++k) q2[4 * i + k] = S.quartets[4 * j + k];
      of2[i] = S.offsets[j];
      sl2[i] = S.qslot[j];
    }
    int64_t npq = 0, nt = 0;
    for (int64_t i = 0; i < n; ++i) {
      for (int k = 0; k < 4; ++k) S.quartets[4 * i + k] = q2[4 * i + k];
      S.offsets[i] = of2[i];
      S.qslot[i] = sl2[i];
      const f12int_ctx::BasisData &B = *batch[sl2[i]]->B;
      S.pq_off[i] = npq;
      npq += (int64_t)B.nprim[q2[4 * i]] * B.nprim[q2[4 * i + 1]] * B.nprim[q2[4 * i + 2]] * B.nprim[q2[4 * i + 3]];
    }
    S.pq_off[n] = npq;
    S.counts[0] = n;
    S.counts[1] = npq;
    int64_t i = 0;
    for (int t = 0; t < kSlots; ++t) {
      S.counts[2 + 2 * t] = nt;
      for (; i < n && items[i].tier == t; ++i)
        for (int sp = 0; sp < items[i].nsplit; ++sp) S.tasks[nt++] = CTask{(int32_t)i, (int16_t)sp, (int16_t)items[i].nsplit};
      S.counts[3 + 2 * t] = nt;
    }
    // copy what this batch uses
    const ClassLists &D = E.dev[cls];
    cudaStream_t st = E.stream;
    const size_t ns = batch.size();
    CK(cudaMemcpyAsync(D.counts, S.counts, sizeof(int64_t) * kCounts, cudaMemcpyHostToDevice, st));
    if (n > 0) {
      CK(cudaMemcpyAsync(D.quartets, S.quartets, sizeof(int32_t) * 4 * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(D.pq_off, S.pq_off, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(D.offsets, S.offsets, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(D.qslot, S.qslot, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(D.tasks, S.tasks, sizeof(CTask) * nt, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(D.views, S.views, sizeof(PairView) * ns, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(D.outs, S.outs, sizeof(double *) * ns, cudaMemcpyHostToDevice, st));
    }
  }
  *E.zstage_count[b] = nzero;
  cudaStream_t st = E.stream;
  CK(cudaMemcpyAsync(E.zero_count, E.zstage_count[b], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (nzero > 0) {
    CK(cudaMemcpyAsync(E.zero_dst, E.zstage_dst[b], sizeof(double *) * nzero, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(E.zero_len, E.zstage_len[b], sizeof(int64_t) * nzero, cudaMemcpyHostToDevice, st));
  }
  CK(cudaGraphLaunch(E.exec, st));
  CK(cudaMemcpyAsync(E.stage_status[b], E.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaMemsetAsync(E.status, 0, sizeof(unsigned), st));
  CK(cudaEventRecord(E.ev[b], st));
  return F12INT_OK;
}

static void engine_worker(f12int_ctx *ctx, Engine *Ep) {
  Engine &E = *Ep;
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(E.mu);
  for (;;) {
    E.cv.wait(lk, [&] { return E.stop || !E.pending.empty(); });
    if (E.pending.empty()) break;   // stop requested and nothing left
    const int b = E.cur;
    E.cur ^= 1;
    // staging buffer b is free once the batch that used it has finished
    if (!E.inflight[b].empty()) {
      lk.unlock();
      cudaEventSynchronize(E.ev[b]);
      lk.lock();
      engine_finish_batch(E, b);
    }
    // admission: take requests while every class fits the batch limits
    std::vector<EngineReq *> batch;
    int64_t nq[7] = {0}, ni[7] = {0}, nt[7] = {0};
    while (!E.pending.empty() && (int64_t)batch.size() < E.scap) {
      EngineReq *R = E.pending.front();
      bool fits = true;
      for (int c = 1; c <= 6; ++c)
        if (nq[c] + R->quartets[c] > E.qcap || ni[c] + R->items[c] > E.icap || nt[c] + R->tasks[c] > E.tcap)
          fits = false;
      if (!fits && !batch.empty()) break;
      for (int c = 1; c <= 6; ++c) {
        nq[c] += R->quartets[c];
        ni[c] += R->items[c];
        nt[c] += R->tasks[c];
      }
      batch.push_back(R);
      E.pending.pop_front();
    }
    int rc = F12INT_OK;
    if (E.graph_dirty) rc = engine_capture(ctx, E);
    for (EngineReq *R : batch) E.tickets[R->ticket].batch = b;
    lk.unlock();
    if (rc == F12INT_OK) rc = engine_launch(ctx, E, batch, b);
    lk.lock();
    for (EngineReq *R : batch) {
      if (rc == F12INT_OK) {
        E.inflight[b].push_back(R->ticket);
      } else {
        TicketState &T = E.tickets[R->ticket];
        T.done = true;
        T.rc = rc;
        T.batch = -1;
      }
      delete R;
    }
    ++E.batches;
  }
}

}  // namespace

static void engine_shutdown(f12int_ctx *ctx) {
  Engine *E = ctx->engine;
  if (!E) return;
  {
    std::lock_guard<std::mutex> lk(E->mu);
    E->stop = true;
  }
  E->cv.notify_all();
  if (E->worker.joinable()) E->worker.join();
  if (E->stream) cudaStreamSynchronize(E->stream);
  for (int c = 1; c <= 6; ++c) lists_free(E->dev[c], false);
  for (int b = 0; b < 2; ++b) {
    for (int c = 1; c <= 6; ++c) lists_free(E->stage[b][c], true);
    cudaFreeHost(E->zstage_dst[b]);
    cudaFreeHost(E->zstage_len[b]);
    cudaFreeHost(E->zstage_count[b]);
    cudaFreeHost(E->stage_status[b]);
    if (E->ev[b]) cudaEventDestroy(E->ev[b]);
  }
  void *ds[] = {E->zero_dst, E->zero_len, E->zero_count, E->status};
  for (void *p : ds)
    if (p) cudaFree(p);
  for (int c = 1; c <= 6; ++c) {
    void *cs[] = {E->keys[c], E->order[c], E->part[c], E->hist[c]};
    for (void *p : cs)
      if (p) cudaFree(p);
    if (E->branch[c]) cudaStreamDestroy(E->branch[c]);
  }
  ctx->used -= std::min(ctx->used, E->bytes);
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->stream) cudaStreamDestroy(E->stream);
  for (EngineReq *R : E->pending) delete R;
  delete E;
  ctx->engine = nullptr;
}

// No request queued or running.
static bool engine_idle(f12int_ctx *ctx) {
  Engine *E = ctx->engine;
  if (!E) return true;
  std::lock_guard<std::mutex> lk(E->mu);
  for (const auto &kv : E->tickets)
    if (!kv.second.done) {
      const int b = kv.second.batch;
      if (b < 0 || cudaEventQuery(E->ev[b]) != cudaSuccess) return false;
    }
  return E->pending.empty();
}

// The captured graph holds the factor's tables by value.
static void engine_factor_changed(f12int_ctx *ctx) {
  if (ctx->engine) {
    std::lock_guard<std::mutex> lk(ctx->engine->mu);
    ctx->engine->graph_dirty = true;
  }
}

extern "C" {

int f12int_batch_limits(f12int_ctx *ctx, int64_t max_quartets, int64_t max_items) {
  if (!ctx || max_quartets < 1 || max_items < 1 || max_quartets > ((int64_t)1 << 30)) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->engine && ctx->engine->ready) return F12INT_EINVAL;   // fixed once the engine runs
  if (!ctx->engine) ctx->engine = new (std::nothrow) Engine();
  if (!ctx->engine) return F12INT_ENOMEM;
  ctx->engine->qcap = max_quartets;
  ctx->engine->icap = max_items;
  return F12INT_OK;
}

// Device memory the one-time primitive bounds of (basis, class) take at most:
// the per-primitive basis's pair data (E and F tables of every primitive
// pair), the diagonal blocks of every primitive pair and the work items of
// one call over them (the buffers of ensure_prim_bounds).
static size_t prim_bounds_bytes(const f12int_ctx *ctx, const f12int_ctx::BasisData &B, int cls) {
  std::vector<int> lp;
  for (int s = 0; s < B.nshell; ++s)
    for (int k = 0; k < B.nprim[s]; ++k) lp.push_back(B.l[s]);
  const size_t np = lp.size();
  size_t pair_data = 0, diag = 0;
  for (size_t a = 0; a < np; ++a)
    for (size_t b = 0; b <= a; ++b) {
      const size_t la = (size_t)lp[a], lb = (size_t)lp[b];
      pair_data += 2 * (6 * (la + 1) * (lb + 1) * (la + lb + 1) + 16) * sizeof(double);
      const size_t nab = (size_t)ncart((int)la) * ncart((int)lb);
      diag += nab * nab * sizeof(double) + 3 * sizeof(int64_t) + 4 * sizeof(int32_t);
    }
  const size_t npairs = np * (np + 1) / 2;
  const size_t nf = (size_t)std::max(1, ctx->tables.nfam[cls == 5 ? 3 : cls]);
  const size_t items = npairs * nf * (sizeof(int) + sizeof(unsigned) + sizeof(double) * kPartPitch);
  return pair_data + diag + items;
}

int f12int_submit(f12int_ctx *ctx, int basis_id, const f12int_request *req, uint64_t *ticket) {
  if (!ctx || !req || !ticket) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size() || !ctx->factor_ready) return F12INT_ENOTREADY;
  if (req->n_quartets < 0 || (req->n_quartets > 0 && (!req->quartets || !req->offsets || !req->out_dev)))
    return F12INT_EINVAL;
  if (req->class_mask == 0 || (req->class_mask >> 6) != 0) return F12INT_EINVAL;
  for (int c = 1; c <= 6; ++c)
    if (((req->class_mask >> (c - 1)) & 1) && !ctx->cls_ok[c]) return F12INT_EDOMAIN;
  if (req->precision != 0 && req->precision != 1) return F12INT_EINVAL;
  if (!(req->schwarz_thresh >= 0.0)) return F12INT_EINVAL;
  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  const int64_t n = req->n_quartets;
  int nclass = 0;
  for (int c = 1; c <= 6; ++c) nclass += (req->class_mask >> (c - 1)) & 1;
  EngineReq *R = new (std::nothrow) EngineReq();
  if (!R) return F12INT_ENOMEM;
  R->basis = basis_id;
  R->B = &B;
  R->mask = req->class_mask;
  R->precision = req->precision;
  R->thresh = req->schwarz_thresh;
  R->out = req->out_dev;
  R->q.assign(req->quartets, req->quartets + 4 * n);
  R->off.assign(req->offsets, req->offsets + (size_t)nclass * n);
  int64_t npq = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *s = &R->q[4 * (size_t)i];
    for (int k = 0; k < 4; ++k)
      if (s[k] < 0 || s[k] >= B.nshell) {
        delete R;
        return F12INT_EINVAL;
      }
    npq += (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]];
  }
  // one-time per (basis, class) work: primitive and shell-pair bounds
  for (int c = 1; c <= 6; ++c) {
    if (!((R->mask >> (c - 1)) & 1)) continue;
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *s = &R->q[4 * (size_t)i];
      BatchPlan bp{};
      const int64_t np = (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]];
      if (!batch_plan(B.l[s[0]], B.l[s[1]], B.l[s[2]], B.l[s[3]], c, np, kTaskFlops / 8, &bp)) {
        delete R;
        return F12INT_EINVAL;
      }
      R->tasks[c] += bp.nsplit;
    }
    // admission by free device memory: the one-time bounds allocate, so a
    // request whose bounds would not fit in what is free now (or in the
    // context's budget) is refused before anything is allocated
    if (B.prim_screen && !B.d_qprim[c]) {
      size_t free_b = 0, total_b = 0;
      const size_t need = prim_bounds_bytes(ctx, B, c);
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
          (need > free_b || (ctx->budget && ctx->used + need > ctx->budget))) {
        delete R;
        return F12INT_ENOMEM;
      }
    }
    int rc = ensure_prim_bounds(ctx, basis_id, c);
    if (rc == F12INT_OK && (R->thresh > 0.0 || R->precision == 1)) rc = ensure_pair_bounds(ctx, basis_id, c);
    if (rc != F12INT_OK) {
      delete R;
      return rc;
    }
    R->quartets[c] = n;
    R->items[c] = npq * ctx->tables.nfam[c == 5 ? 3 : c];
  }
  Engine *E = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->engine) ctx->engine = new (std::nothrow) Engine();
    E = ctx->engine;
    if (!E) {
      delete R;
      return F12INT_ENOMEM;
    }
    if (!E->ready) {
      CK(cudaSetDevice(ctx->device));
      int rc = engine_init(ctx, *E);
      if (rc != F12INT_OK) {
        delete R;
        return rc;
      }
      E->worker = std::thread(engine_worker, ctx, E);
    }
  }
  for (int c = 1; c <= 6; ++c)
    if (R->quartets[c] > E->qcap || R->items[c] > E->icap || R->tasks[c] > 4 * E->qcap) {
      delete R;
      return F12INT_ENOMEM;   // larger than one batch: not admitted
    }
  {
    std::lock_guard<std::mutex> lk(E->mu);
    R->ticket = E->next_ticket++;
    *ticket = R->ticket;
    E->tickets[R->ticket] = TicketState{};
    E->pending.push_back(R);
  }
  E->cv.notify_one();
  return F12INT_OK;
}

int f12int_poll(f12int_ctx *ctx, uint64_t ticket, int64_t timeout_us, int *done) {
  if (!ctx || !done || timeout_us < 0) return F12INT_EINVAL;
  Engine *E = ctx->engine;
  if (!E) return F12INT_EINVAL;
  *done = 0;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(E->mu);
      auto it = E->tickets.find(ticket);
      if (it == E->tickets.end()) return F12INT_EINVAL;
      if (!it->second.done && it->second.batch >= 0) {
        const int b = it->second.batch;
        bool mine = false;
        for (uint64_t t : E->inflight[b]) mine |= (t == ticket);
        if (mine && cudaEventQuery(E->ev[b]) == cudaSuccess) engine_finish_batch(*E, b);
      }
      if (it->second.done) {
        const int rc = it->second.rc;
        E->tickets.erase(it);
        *done = 1;
        return rc;
      }
    }
    if (std::chrono::steady_clock::now() >= deadline) return timeout_us > 0 ? F12INT_ETIMEOUT : F12INT_OK;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int f12int_batch_autotune(f12int_ctx *ctx, int basis_id, const int32_t *quartets, int64_t n, uint32_t class_mask,
                          double *report) {
  if (!ctx || !quartets || n <= 0 || class_mask == 0 || (class_mask >> 6) != 0) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size() || !ctx->factor_ready) return F12INT_ENOTREADY;
  if (!engine_idle(ctx)) return F12INT_EINVAL;
  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  std::vector<int64_t> off((size_t)n);
  int64_t tot = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *s = quartets + 4 * i;
    for (int k = 0; k < 4; ++k)
      if (s[k] < 0 || s[k] >= B.nshell) return F12INT_EINVAL;
    off[i] = tot;
    tot += (int64_t)ncart(B.l[s[0]]) * ncart(B.l[s[1]]) * ncart(B.l[s[2]]) * ncart(B.l[s[3]]);
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->engine) ctx->engine = new (std::nothrow) Engine();
    if (!ctx->engine) return F12INT_ENOMEM;
  }
  double *out = nullptr;
  int rc = dalloc(ctx, &out, sizeof(double) * (size_t)tot);
  if (rc != F12INT_OK) return rc;
  const double targets[4] = {kTaskFlops / 8, kTaskFlops * 0.3, kTaskFlops, kTaskFlops * 4};
  const int divs[2] = {1, 2};
  // one request of class c, alone in its batch; seconds from submit to done
  auto run = [&](int c, double *sec) -> int {
    f12int_request rq{n, quartets, 1u << (c - 1), 0, 0.0, out, off.data()};
    uint64_t t = 0;
    const auto t0 = std::chrono::steady_clock::now();
    int r = f12int_submit(ctx, basis_id, &rq, &t);
    int done = 0;
    // wait until the request is done (a 100 ms wait that runs out returns
    // F12INT_ETIMEOUT with done = 0: keep waiting)
    while ((r == F12INT_OK || r == F12INT_ETIMEOUT) && !done) r = f12int_poll(ctx, t, 100000, &done);
    *sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return r;
  };
  for (int c = 1; c <= 6 && rc == F12INT_OK; ++c) {
    if (!((class_mask >> (c - 1)) & 1)) continue;
    double best = 1e300, bt = kTaskFlops;
    int bd = 1;
    for (double tg : targets)
      for (int dv : divs) {
        {
          std::lock_guard<std::mutex> lk(ctx->engine->mu);
          ctx->engine->task_target[c] = tg;
          ctx->engine->items_div[c] = dv;
          ctx->engine->graph_dirty = true;
        }
        double t1 = 0.0, t2 = 0.0;
        rc = run(c, &t1);   // first run after a change includes the graph capture
        if (rc == F12INT_OK) rc = run(c, &t2);
        if (rc != F12INT_OK) break;
        if (t2 < best) {
          best = t2;
          bt = tg;
          bd = dv;
        }
      }
    if (rc != F12INT_OK) break;
    {
      std::lock_guard<std::mutex> lk(ctx->engine->mu);
      ctx->engine->task_target[c] = bt;
      ctx->engine->items_div[c] = bd;
      ctx->engine->graph_dirty = true;
    }
    if (report) {
      report[3 * (c - 1)] = bt;
      report[3 * (c - 1) + 1] = bd;
      report[3 * (c - 1) + 2] = best;
    }
  }
  // the sample's output may be freed only once no batch writes it any more
  // (an error above can leave one in flight): bounded wait, else keep it
  bool idle = engine_idle(ctx);
  for (int k = 0; k < 6000 && !idle; ++k) {
    std::this_thread::sleep_for(std::chrono::milliseconds(10));
    idle = engine_idle(ctx);
  }
  if (idle) dfree(ctx, out, sizeof(double) * (size_t)tot);
  return idle ? rc : F12INT_ETIMEOUT;
}

int f12int_set_fp32_below(f12int_ctx *ctx, double bound) {
  if (!ctx || !(bound >= 0.0)) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->engine) ctx->engine = new (std::nothrow) Engine();
  if (!ctx->engine) return F12INT_ENOMEM;
  std::lock_guard<std::mutex> lk2(ctx->engine->mu);
  ctx->engine->fp32_below = bound;
  return F12INT_OK;
}

int f12int_batch_stats(f12int_ctx *ctx, int64_t *stats) {
  if (!ctx || !stats) return F12INT_EINVAL;
  Engine *E = ctx->engine;
  if (!E) {
    stats[0] = stats[1] = stats[2] = 0;
    return F12INT_OK;
  }
  std::lock_guard<std::mutex> lk(E->mu);
  stats[0] = E->batches;
  stats[1] = E->requests_done;
  stats[2] = (int64_t)E->pending.size();
  return F12INT_OK;
}

}  // extern "C"
