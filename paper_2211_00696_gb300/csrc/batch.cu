// Batched apply over many plans (uneven sizes) x right-hand sides: every stage of
// Algorithm 1 + Algorithm 6 for all of them runs as one grouped persistent launch, and the
// whole sequence is one CUDA graph.  An optional empirical autotuner picks the tile shape
// (K chunk of 32 or 64), the job order within a pass (as built, or largest first) and the
// grid size on the first apply, timing each candidate with CUDA events on the caller's stream.
#include <algorithm>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "batch.h"
#include "checked.cuh"
#include "plan.h"

using namespace phikron;


struct phikron_batch_s {
  Profiler prof;   // launches of the applies (timing: phikron_batch_profile_begin/end)
  std::vector<const Plan*> plans;
  int nrhs = 1;
  bool half = false;
  int device = 0;
  std::vector<void*> work;
  size_t work_bytes = 0;
  std::vector<std::unique_ptr<Seq>> cand;
  std::vector<SeqConfig> cfgs;
  std::vector<float> cand_ms;
  int chosen = 0;
  bool tuned = false;
  ~phikron_batch_s() {
    cand.clear();
    for (void* p : work) device_free(p);
  }
};

namespace {

int walloc(phikron_batch_s& B, void** p, size_t bytes) {
  PK_RET(device_malloc(p, bytes ? bytes : 16, "phikron_batch_create"));
  B.work.push_back(*p);
  B.work_bytes += bytes;
  return PHIKRON_OK;
}

PtrArgs make_args(const phikron_batch_s& B, const double* const* V, double* const* Out) {
  PtrArgs a{};
  a.n = 2 * (int)B.plans.size();
  for (size_t i = 0; i < B.plans.size(); ++i) {
    a.p[2 * i] = const_cast<double*>(V[i]);
    a.p[2 * i + 1] = Out[i];
  }
  return a;
}

}  // namespace

extern "C" {

int phikron_batch_create(phikron_batch_t* out, int count, const phikron_plan_t* plans, int nrhs, int half_step,
                         int autotune) {
  clear_error();
  if (!out || !plans || count < 1 || count > MAX_PTRS / 2 || nrhs < 1) {
    set_error("phikron_batch_create: need 1 <= count <= 64 plans and nrhs >= 1");
    return PHIKRON_EINVAL;
  }
  *out = nullptr;
  std::unique_ptr<phikron_batch_s> B(alloc_fault() ? nullptr : new (std::nothrow) phikron_batch_s());
  if (!B) {
    set_error("phikron_batch_create: host allocation failed");
    return PHIKRON_ENOMEM;
  }
  B->nrhs = nrhs;
  B->half = half_step != 0;
  int slices = -1;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) {
      set_error("phikron_batch_create: NULL plan");
      return PHIKRON_EINVAL;
    }
    const Plan& P = plans[i]->impl;
    if (P.opts.precision != PHIKRON_PREC_OZAKI_BF16 || !P.mixed) {
      set_error("phikron_batch_create: every plan must use PHIKRON_PREC_OZAKI_BF16");
      return PHIKRON_ENOTSUP;
    }
    if (P.PN != P.N) {
      set_error("phikron_batch_create: batched plans need every n[d] a multiple of 16 (no padding)");
      return PHIKRON_ENOTSUP;
    }
    const int ks = mixed_slices(P);
    if (slices >= 0 && ks != slices) {
      set_error("phikron_batch_create: every plan must use the same digit-slice count");
      return PHIKRON_EINVAL;
    }
    slices = ks;
    if (B->half && !P.opts.half_step) {
      set_error("phikron_batch_create: half_step outputs need plans made with opts.half_step");
      return PHIKRON_EINVAL;
    }
    if (i > 0 && P.opts.device != plans[0]->impl.opts.device) {
      set_error("phikron_batch_create: every plan must live on the same device");
      return PHIKRON_EINVAL;
    }
    B->plans.push_back(&P);
  }
  B->device = plans[0]->impl.opts.device;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    set_error("cudaGetDevice failed");
    return PHIKRON_ECUDA;
  }
  if (B->device >= 0 && B->device != prev) cudaSetDevice(B->device);
  int rc = PHIKRON_OK;
  do {
    // work buffers per unit
    std::vector<SeqUnit> units;
    for (int i = 0; i < count && rc == PHIKRON_OK; ++i) {
      const Plan& P = *B->plans[i];
      const int nv = std::max(P.m + 2, std::max(P.p, 1));
      for (int r = 0; r < nrhs && rc == PHIKRON_OK; ++r) {
        SeqUnit u{};
        u.plan = &P;
        u.inst = i;
        u.rhs = r;
        void *w1, *w2, *y, *yn;
        if (r == 0) {  // the first right-hand side reuses the plan's own work buffers
          w1 = P.dW1;
          w2 = P.dW2;
          y = P.dY;
          yn = P.dYn;
        } else {
          if ((rc = walloc(*B, &w1, sizeof(float2) * (size_t)nv * P.N)) != PHIKRON_OK) break;
          if ((rc = walloc(*B, &w2, sizeof(float2) * (size_t)nv * P.N)) != PHIKRON_OK) break;
          if ((rc = walloc(*B, &y, sizeof(float2) * (size_t)std::max(P.p, 1) * P.N)) != PHIKRON_OK) break;
          if ((rc = walloc(*B, &yn, sizeof(float2) * (size_t)std::max(P.p, 1) * P.N)) != PHIKRON_OK) break;
        }
        u.W1 = (float2*)w1;
        u.W2 = (float2*)w2;
        u.Y = (float2*)y;
        u.Yn = (float2*)yn;
        units.push_back(u);
      }
    }
    if (rc != PHIKRON_OK) break;
    int nsm = 148;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // candidate launch shapes
    std::vector<SeqConfig> cfgs;
    // kernel variants: 2 = double-buffered (where every n >= 64), 1 = warp-specialised,
    // 0 = single-role; the default first, the others as autotuner candidates
    const int v0 = mode_kernel_db_default() ? 2 : (mode_kernel_ws_default() ? 1 : 0);
    std::vector<int> variants = {v0};
    for (int v : {2, 1}) if (v != v0) variants.push_back(v);
    for (int var : variants) {
      for (int sub : {1, 2}) {
        if (sub == 2 && (slices != 3 || var != 0)) continue;  // 64-wide chunks: single-role kernel only
        for (bool bf : {false, true}) {
          for (int g : {nsm, (3 * nsm) / 4}) {
            SeqConfig c;
            c.half = B->half;
            c.slices = slices;
            c.sub = sub;
            c.grid = g;
            c.big_first = bf;
            c.graph = true;
            c.ws = var >= 1;
            c.db = var == 2;
            c.fuse = fused_weights_default();
            c.rr = raw_ring_default();
            cfgs.push_back(c);
            if (!autotune) break;
          }
          if (!autotune) break;
        }
        if (!autotune) break;
      }
      if (!autotune) break;
    }
    for (const SeqConfig& c : cfgs) {
      std::unique_ptr<Seq> S(new Seq());
      std::vector<SeqUnit> us = units;
      if ((rc = seq_build(*S, us, count, c)) != PHIKRON_OK) break;
      B->cand.push_back(std::move(S));
      B->cfgs.push_back(c);
    }
    B->tuned = (B->cand.size() <= 1);
  } while (0);
  if (B->device >= 0 && B->device != prev) cudaSetDevice(prev);
  if (rc != PHIKRON_OK) return rc;
  *out = B.release();
  return PHIKRON_OK;
}

int phikron_batch_apply(phikron_batch_t b, const double* const* V, double* const* Out, void* stream) {
  clear_error();
  if (!b || !V || !Out) {
    set_error("phikron_batch_apply: NULL argument");
    return PHIKRON_EINVAL;
  }
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (!V[i] || !Out[i]) {
      set_error("phikron_batch_apply: NULL vector pointer");
      return PHIKRON_EINVAL;
    }
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    set_error("cudaGetDevice failed");
    return PHIKRON_ECUDA;
  }
  if (b->device >= 0 && b->device != prev) cudaSetDevice(b->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<chk::Range> rr;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const Plan& P = *b->plans[i];
    rr.push_back({V[i], sizeof(double) * (size_t)P.N * b->nrhs});
    rr.push_back({Out[i], sizeof(double) * (size_t)P.N * (P.p + 1) * (b->half ? 2 : 1) * b->nrhs});
  }
  chk::CallScope cs(st, rr.data(), (int)rr.size());
  if (cs.rc != PHIKRON_OK) {
    if (b->device >= 0 && b->device != prev) cudaSetDevice(prev);
    return cs.rc;
  }
  const PtrArgs args = make_args(*b, V, Out);
  int rc = PHIKRON_OK;
  if (!b->tuned) {
    // first apply: time every candidate (each run overwrites Out with the same result)
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    b->cand_ms.assign(b->cand.size(), 0.f);
    float best = 1e30f;
    for (size_t c = 0; c < b->cand.size() && rc == PHIKRON_OK; ++c) {
      rc = seq_run(*b->cand[c], args, st);  // warm-up
      for (int rep = 0; rep < 2 && rc == PHIKRON_OK; ++rep) {
        cudaEventRecord(e0, st);
        rc = seq_run(*b->cand[c], args, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->cand_ms[c] = (rep == 0) ? ms : std::min(b->cand_ms[c], ms);
      }
      if (b->cand_ms[c] < best) {
        best = b->cand_ms[c];
        b->chosen = (int)c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned = true;
  }
  if (rc == PHIKRON_OK) {
    ProfScope ps(&b->prof);
    rc = seq_run(*b->cand[b->chosen], args, st);
  }
  if (b->device >= 0 && b->device != prev) cudaSetDevice(prev);
  return rc;
}

int phikron_batch_profile_begin(phikron_batch_t b, int max_timed) {
  clear_error();
  if (!b || max_timed < 0) {
    set_error("phikron_batch_profile_begin: bad arguments");
    return PHIKRON_EINVAL;
  }
  return profiler_begin(b->prof, max_timed);
}

int phikron_batch_profile_end(phikron_batch_t b, phikron_profile* out) {
  clear_error();
  if (!b || !out) {
    set_error("phikron_batch_profile_end: NULL argument");
    return PHIKRON_EINVAL;
  }
  *out = phikron_profile{};
  return profiler_end(b->prof, out);
}

int phikron_batch_get_info(phikron_batch_t b, phikron_batch_info* info) {
  clear_error();
  if (!b || !info) {
    set_error("phikron_batch_get_info: NULL argument");
    return PHIKRON_EINVAL;
  }
  const Seq& S = *b->cand[b->chosen];
  const SeqConfig& c = b->cfgs[b->chosen];
  info->units = (int)(b->plans.size()) * b->nrhs;
  info->launches = (int)S.steps.size();
  info->mode_jobs = (long long)S.njobs_mode;
  info->graph = S.exec != nullptr;
  info->k_chunk = 32 * c.sub;
  info->big_first = c.big_first ? 1 : 0;
  info->grid = c.grid;
  info->candidates = (int)b->cand.size();
  info->tuned = b->tuned ? 1 : 0;
  info->best_ms = b->cand_ms.empty() ? 0.0 : b->cand_ms[b->chosen];
  size_t bytes = b->work_bytes;
  for (const auto& s : b->cand) bytes += s->device_bytes;
  info->device_bytes = bytes;
  info->ws_kernel = c.db ? 2 : (c.ws ? 1 : 0);
  return PHIKRON_OK;
}

int phikron_batch_check_status(phikron_batch_t b) {
  clear_error();
  if (!b) {
    set_error("phikron_batch_check_status: NULL batch");
    return PHIKRON_EINVAL;
  }
  PK_TRY_CUDA(cudaDeviceSynchronize());
  PK_RET(chk::status());   // bounds-checked build: a recorded out-of-range access
  for (auto& s : b->cand) {
    int st = 0;
    PK_RET(seq_status(*s, &st));
    if (st != 0) {
      set_error("a bounded device wait expired during an earlier batched apply");
      return st;
    }
  }
  return PHIKRON_OK;
}

void phikron_batch_destroy(phikron_batch_t b) { delete b; }

}  // extern "C"
