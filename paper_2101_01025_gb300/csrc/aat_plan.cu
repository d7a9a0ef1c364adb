// aat_plan.cu -- batched execution of many independent products of a matrix
// by its adjoint: one plan built once, executed as one CUDA graph launch.
//
// At creation the plan sorts its problems:
//   * F_p problems whose recursion depth is 0 (the leaves are the whole
//     product) join one batch: one batched split kernel writes every digit
//     plane set, and ONE persistent tensor-core leaf launch walks a single
//     tile list spanning all of them (per-problem tensor maps, group tables
//     and outputs live in device tables), heaviest tiles first;
//   * complex A A^H problems (Algorithm 2, 2M) join a second batch: one
//     split, ONE persistent FP32 leaf launch over the H and G tiles of all
//     of them, one combine and one diagonal launch, on a side stream beside
//     the F_p batch;
//   * every other problem (recursive F_p products, complex A A^T) runs its
//     own sequence of launches.
// The other problems are spread round robin over up to kBranches side
// streams, each with its own workspace region, so that the small launches of
// different problems share the SMs; the batch runs on the main stream beside
// them.  The plan owns its workspace, runs everything once eagerly (so every
// cache and kernel attribute exists), then captures the same fork/join
// sequence into a CUDA graph.  aat_plan_execute launches that graph on the
// caller's stream: no allocation, no host synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/aat.h"
#include "common.cuh"

namespace aat {

constexpr int kBranches = 16;

struct Plan {
  int dev = 0;
  cudaStream_t st = nullptr;
  std::vector<cudaStream_t> side;  // one per branch
  std::vector<cudaEvent_t> ev;     // fork event + one join event per branch
  size_t region = 0;               // bytes of one branch's workspace region
  void *ws = nullptr;
  size_t ws_size = 0;
  std::vector<aat_problem_t> probs;
  std::vector<int> solo;          // problems run on their own
  std::vector<int> batched;       // F_p problems in the batched leaf launch
  std::vector<int> cbatched;      // complex A A^H problems in the complex batch
  CBatch cb;
  cudaStream_t cb_st = nullptr;   // the complex batch's stream
  cudaEvent_t cb_ev[2] = {nullptr, nullptr};  // its fork and join
  std::vector<TcLeafArgs> leaf_args;
  std::vector<ModP> leaf_mods;
  SplitDesc *split_dev = nullptr;
  int nsplit = 0;
  int split_blocks = 0;
  double split_bytes = 0.0;
  LeafBatch leaf;
  size_t solo_off = 0;            // workspace offset of the shared region
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static int enqueue(Plan &P, cudaStream_t st) {
  cudaError_t ce;
  if (!P.cbatched.empty()) {  // the complex batch on its own stream
    if ((ce = cudaEventRecord(P.cb_ev[0], st)) != cudaSuccess ||
        (ce = cudaStreamWaitEvent(P.cb_st, P.cb_ev[0], 0)) != cudaSuccess ||
        (ce = cbatch_launch(P.cb, P.cb_st)) != cudaSuccess ||
        (ce = cudaEventRecord(P.cb_ev[1], P.cb_st)) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  const int nb = (int)P.side.size();
  if (nb > 0) {  // fork the side branches off the main stream
    if ((ce = cudaEventRecord(P.ev[0], st)) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    for (int b = 0; b < nb; ++b)
      if ((ce = cudaStreamWaitEvent(P.side[b], P.ev[0], 0)) != cudaSuccess)
        return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  for (size_t q = 0; q < P.solo.size(); ++q) {
    const int b = (int)(q % (size_t)nb);
    const aat_problem_t &pr = P.probs[P.solo[q]];
    char *region = (char *)P.ws + P.solo_off + (size_t)b * P.region;
    int e;
    if (pr.kind == AAT_KIND_MODP)
      e = modp_run((const int32_t *)pr.A, pr.n, pr.k, pr.lda, pr.p, (int32_t *)pr.C, pr.ldc,
                   pr.flags, P.side[b], region, false, nullptr);
    else
      e = complex_run(pr.kind == AAT_KIND_AAH ? 0 : 2, pr.A, pr.n, pr.k, pr.lda, pr.C, pr.ldc,
                      pr.flags, P.side[b], region, false, nullptr);
    if (e) return e;
  }
  if (P.nsplit > 0) {
    if ((ce = launch_split_batch(P.split_dev, P.nsplit, P.split_blocks, P.split_bytes, st)) !=
        cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    if ((ce = leaf_tc_batch_launch(P.leaf, st)) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  for (int b = 0; b < nb; ++b) {  // join
    if ((ce = cudaEventRecord(P.ev[1 + b], P.side[b])) != cudaSuccess ||
        (ce = cudaStreamWaitEvent(st, P.ev[1 + b], 0)) != cudaSuccess)
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  if (!P.cbatched.empty() && (ce = cudaStreamWaitEvent(st, P.cb_ev[1], 0)) != cudaSuccess)
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  return AAT_OK;
}

static void destroy(Plan *P) {
  if (!P) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(P->dev);
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  leaf_tc_batch_free(&P->leaf);
  cbatch_free(&P->cb);
  for (cudaEvent_t e : P->cb_ev)
    if (e) cudaEventDestroy(e);
  if (P->cb_st) cudaStreamDestroy(P->cb_st);
  if (P->split_dev) cudaFree(P->split_dev);
  if (P->ws) cudaFree(P->ws);
  for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
  for (cudaStream_t s : P->side) cudaStreamDestroy(s);
  if (P->st) cudaStreamDestroy(P->st);
  cudaSetDevice(cur);
  delete P;
}

static int create(const aat_problem_t *probs, int count, Plan **out) {
  if (!out || count < 0 || (count > 0 && !probs)) return report_error(AAT_EINVAL, "bad arguments");
  int e = check_gb300();
  if (e) return e;
  Plan *P = new Plan;
  cudaGetDevice(&P->dev);
  P->probs.assign(probs, probs + count);
  auto r256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // validate and sort the problems; size the batch's planes
  size_t batch_bytes = 0, solo_bytes = 0;
  std::vector<size_t> plane_off(count, 0);
  for (int i = 0; i < count; ++i) {
    const aat_problem_t &q = P->probs[i];
    const bool fp = q.kind == AAT_KIND_MODP;
    if (q.kind != AAT_KIND_MODP && q.kind != AAT_KIND_AAH && q.kind != AAT_KIND_AAT_C) {
      destroy(P);
      return report_error(AAT_EINVAL, "unknown problem kind");
    }
    if (q.n <= 0 || q.k <= 0 || !q.A || !q.C || q.lda < q.k || q.ldc < q.n) {
      destroy(P);
      return report_error(AAT_EINVAL, ("bad sizes, strides or pointers in problem " +
                                        std::to_string(i)).c_str());
    }
    if (fp) {
      if ((e = check_prime_arg(q.p))) {
        destroy(P);
        return e;
      }
      const bool tc = (q.flags & AAT_LEAF_MASK) == AAT_LEAF_TC;
      const bool extra = (q.flags & AAT_ZERO_UPPER) != 0;
      if (tc && !extra && modp_levels(q.n, q.k, q.p, q.flags) == 0) {
        const DigitSpec ds = digits_for_problem(q.n, q.k, q.p, q.flags);
        const Planes pl = planes_layout(ds, q.n, q.k);
        plane_off[i] = batch_bytes;
        batch_bytes += r256((size_t)pl.L * pl.rows * pl.kstride * 2);
        P->batched.push_back(i);
        continue;
      }
    }
    if (q.kind == AAT_KIND_AAH) {
      const uint32_t prec = q.flags & AAT_C_PREC_MASK;
      if (prec != AAT_C_FP32 && prec != AAT_C_BF16X3 && prec != AAT_C_BF16) {
        destroy(P);
        return report_error(AAT_EUNSUPPORTED, "unknown precision");
      }
      P->cbatched.push_back(i);
      continue;
    }
    size_t need = 0;
    if (fp)
      e = modp_run((const int32_t *)q.A, q.n, q.k, q.lda, q.p, (int32_t *)q.C, q.ldc, q.flags,
                   nullptr, nullptr, true, &need);
    else
      e = complex_run(q.kind == AAT_KIND_AAH ? 0 : 2, q.A, q.n, q.k, q.lda, q.C, q.ldc, q.flags,
                      nullptr, nullptr, true, &need);
    if (e) {
      destroy(P);
      return e;
    }
    solo_bytes = std::max(solo_bytes, need);
    P->solo.push_back(i);
  }
  const int nb = std::min<int>(kBranches, (int)P->solo.size());
  std::vector<CBInput> cb_in;
  for (int i : P->cbatched) {
    const aat_problem_t &q = P->probs[i];
    cb_in.push_back(CBInput{(const float2 *)q.A, q.lda, q.n, q.k, (float2 *)q.C, q.ldc, q.flags, 1});
  }
  const size_t cb_off = r256(batch_bytes);
  const size_t cb_bytes = r256(cbatch_workspace(cb_in.data(), (int)cb_in.size()));
  P->region = r256(solo_bytes);
  P->solo_off = cb_off + cb_bytes;
  P->ws_size = P->solo_off + (size_t)nb * P->region + 256;
  cudaError_t ce;
  if ((ce = cudaMalloc(&P->ws, P->ws_size)) != cudaSuccess) {
    cudaGetLastError();
    destroy(P);
    return report_error(AAT_ENOMEM, "plan workspace");
  }
  if ((ce = cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking)) != cudaSuccess) {
    destroy(P);
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  for (int b = 0; b < nb; ++b) {
    cudaStream_t s2 = nullptr;
    if ((ce = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking)) != cudaSuccess) {
      destroy(P);
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    }
    P->side.push_back(s2);
  }
  for (int b = 0; b < (nb ? nb + 1 : 0); ++b) {
    cudaEvent_t ev = nullptr;
    if ((ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
      destroy(P);
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    }
    P->ev.push_back(ev);
  }
  // the complex batch
  if (!P->cbatched.empty()) {
    if ((ce = cudaStreamCreateWithFlags(&P->cb_st, cudaStreamNonBlocking)) != cudaSuccess ||
        (ce = cudaEventCreateWithFlags(&P->cb_ev[0], cudaEventDisableTiming)) != cudaSuccess ||
        (ce = cudaEventCreateWithFlags(&P->cb_ev[1], cudaEventDisableTiming)) != cudaSuccess ||
        (ce = cbatch_build(cb_in.data(), (int)cb_in.size(), (char *)P->ws + cb_off, &P->cb)) !=
            cudaSuccess) {
      destroy(P);
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    }
  }
  // the batch: split descriptors and leaf tables
  if (!P->batched.empty()) {
    std::vector<SplitDesc> sd;
    for (int i : P->batched) {
      const aat_problem_t &q = P->probs[i];
      const DigitSpec ds = digits_for_problem(q.n, q.k, q.p, q.flags);
      Planes pl = planes_layout(ds, q.n, q.k);
      pl.ptr = (__nv_bfloat16 *)((char *)P->ws + plane_off[i]);
      SplitDesc d;
      d.X = (const int32_t *)q.A;
      d.ldx = q.lda;
      d.rows = q.n;
      d.cols = q.k;
      d.m = make_modp(q.p);
      d.b = ds.b;
      d.P = pl;
      sd.push_back(d);
      P->split_bytes += (double)q.n * q.k * (4.0 + 2.0 * pl.L);
      TcLeafArgs a;
      std::memset(&a, 0, sizeof(a));
      a.x = a.y = pl;
      a.dx = a.dy = ds;
      a.M = a.N = q.n;
      a.K = q.k;
      a.out = (int32_t *)q.C;
      a.ldo = q.ldc;
      a.lower = 1;
      a.lin = lin_of(1, 0, q.p);
      a.exact_bits = 24;
      P->leaf_args.push_back(a);
      P->leaf_mods.push_back(d.m);
    }
    P->nsplit = (int)sd.size();
    P->split_blocks = split_batch_blocks(sd.data(), P->nsplit);
    if (P->split_blocks < 0) {
      destroy(P);
      return report_error(AAT_ERANGE, "batch too large for one split launch");
    }
    if ((ce = cudaMalloc(&P->split_dev, sizeof(SplitDesc) * sd.size())) != cudaSuccess ||
        (ce = cudaMemcpy(P->split_dev, sd.data(), sizeof(SplitDesc) * sd.size(),
                         cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ce = leaf_tc_batch_build(P->leaf_args.data(), P->leaf_mods.data(),
                                  (int)P->leaf_args.size(), &P->leaf)) != cudaSuccess) {
      destroy(P);
      return report_error(AAT_ECUDA, cudaGetErrorString(ce));
    }
  }
  // eager run (creates every cache the captured launches use), then capture
  if ((e = enqueue(*P, P->st))) {
    destroy(P);
    return e;
  }
  if ((ce = cudaStreamSynchronize(P->st)) != cudaSuccess) {
    destroy(P);
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  if ((ce = cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
    destroy(P);
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  e = enqueue(*P, P->st);
  cudaGraph_t g = nullptr;
  ce = cudaStreamEndCapture(P->st, &g);
  if (e || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    destroy(P);
    return e ? e : report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  P->graph = g;
  if ((ce = cudaGraphInstantiate(&P->exec, g, 0)) != cudaSuccess) {
    destroy(P);
    return report_error(AAT_ECUDA, cudaGetErrorString(ce));
  }
  *out = P;
  return AAT_OK;
}

}  // namespace aat

using namespace aat;

struct aat_plan {
  Plan *p;
};

extern "C" {

AAT_API int aat_plan_create(const aat_problem_t *probs, int count, aat_plan_t **plan) {
  if (!plan) return report_error(AAT_EINVAL, "null plan");
  *plan = nullptr;
  Plan *P = nullptr;
  int e = create(probs, count, &P);
  if (e) return e;
  *plan = new aat_plan{P};
  return AAT_OK;
}

AAT_API int aat_plan_execute(aat_plan_t *plan, void *stream) {
  if (!plan || !plan->p || !plan->p->exec) return report_error(AAT_EINVAL, "null plan");
  cudaError_t ce = cudaGraphLaunch(plan->p->exec, (cudaStream_t)stream);
  return ce == cudaSuccess ? AAT_OK : report_error(AAT_ECUDA, cudaGetErrorString(ce));
}

AAT_API int aat_plan_info(const aat_plan_t *plan, int *batched, int *solo, size_t *workspace) {
  if (!plan || !plan->p) return report_error(AAT_EINVAL, "null plan");
  if (batched) *batched = (int)(plan->p->batched.size() + plan->p->cbatched.size());
  if (solo) *solo = (int)plan->p->solo.size();
  if (workspace) *workspace = plan->p->ws_size;
  return AAT_OK;
}

AAT_API void aat_plan_destroy(aat_plan_t *plan) {
  if (!plan) return;
  if (plan->p) {
    cudaDeviceSynchronize();
    destroy(plan->p);
  }
  delete plan;
}

}  // extern "C"
