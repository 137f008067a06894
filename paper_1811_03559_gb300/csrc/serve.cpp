// Serving engine of libspike.so (spike_serve.h): a catalogue of banded matrices, their
// factorizations kept resident in device memory under a byte budget (least recently
// used, or lowest greedy-dual size-frequency priority, evicted first), and workers that
// each own one host thread and one CUDA stream.
//
// A factorization is reused for every later request on its matrix, N and T alike
// (Sec. 4 reuses the factors of Sec. 2 for the transpose solve).  Waiting requests
// with the same (matrix, trans, precision) are merged into one multi-column solve:
// the factors and spike tips are then read once for all of them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "spike.h"
#include "spike_serve.h"
#include "internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void sleep_us(int us) {
  if (us > 0) std::this_thread::sleep_for(std::chrono::microseconds(us));
}

struct Req {
  int64_t mid = 0;
  const double *F = nullptr;
  double *X = nullptr;
  int nrhs = 0;
  char trans = 'N';
  int prec = 0;
  double t_submit = 0.0, t_done = 0.0;
  int status = 0;
  bool done = false;
};

// One factorization of a matrix (precision 0 = FP64, 1 = mixed).
struct Fac {
  spike_handle h = nullptr;
  int64_t bytes = 0;      // counted against the budget (a reservation while factoring)
  uint64_t last_use = 0;  // LRU clock
  bool resident = false;  // factored and held
  bool busy = false;      // a worker is factoring or solving with it
  double cost_s = 0.0;    // wall time of its last factorization (SPIKE_SERVE_EVICT_COST)
  int64_t uses = 0;       // solves served since it was factored
  double prio = 0.0;      // greedy-dual priority: L + uses * cost_s / bytes
};

struct Mat {
  const double *band = nullptr;
  int64_t ldab = 0, n = 0;
  int kl = 0, ku = 0, pivot = 0, p = 1;
  bool host = true;
  Fac fac[2];
};

// Per-worker device buffers: solve workspace and the merged right-hand sides.
struct WorkerBuf {
  char *ws = nullptr;
  int64_t ws_bytes = 0;
  double *fb = nullptr;
  int64_t fb_bytes = 0;
};

}  // namespace

struct spike_server_s {
  spike_server_config cfg;
  int dev = 0;
  int sms = 152;
  int batch_systems = 1;  // most matrices per solve (1: one matrix per solve)
  int policy = SPIKE_SERVE_EVICT_LRU;
  double gd_L = 0.0;      // greedy-dual inflation value: priority of the last evicted factorization
  bool dry = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::unordered_map<int64_t, Mat> mats;
  std::deque<Req> reqs;  // index = request id (deque: stable references)
  std::deque<int64_t> pending;
  std::vector<std::thread> th;
  std::vector<cudaStream_t> st;
  std::vector<WorkerBuf> wb;
  bool stop = false;
  int64_t used = 0, peak = 0;
  uint64_t tick = 0;
  int running = 0;  // workers between taking a batch and finishing it
  int waiting = 0;  // of those, workers blocked in admit()
  int64_t batches = 0, rhs = 0, nfact = 0, nevict = 0, nwait = 0, failed = 0, completed = 0, multi = 0;
  int max_batch = 0, max_systems = 0;
  double t_first = -1.0, t_last = 0.0;
  std::vector<double> lat;
  // SPIKE_SERVE_TUNED: fastest worker count per size class (floor(log2 n), k); classes being tuned
  std::map<std::pair<int, int>, int> tuned;
  std::set<std::pair<int, int>> tuning;
  int64_t greplays = 0;  // SPIKE_SERVE_GRAPHS: solves replayed from graphs
  std::string last_error;  // CUDA error text of the last failed request (worker threads' own)
};

namespace {

using Lock = std::unique_lock<std::mutex>;

void account(spike_server_s *S, int64_t delta) {
  S->used += delta;
  S->peak = std::max(S->peak, S->used);
}

// Which of two idle factorizations leaves first under the server's policy.
bool evict_before(const spike_server_s *S, const Fac &a, const Fac &b) {
  if (S->policy == SPIKE_SERVE_EVICT_COST && a.prio != b.prio) return a.prio < b.prio;
  return a.last_use < b.last_use;
}

// Make room for `bytes` more device bytes: evict factorizations that no worker is using
// (least recently used first, or lowest greedy-dual priority first).  Waits while another
// worker that is not itself waiting holds memory that it will release; returns false when
// the bytes cannot fit (so two workers never wait on each other).
bool admit(spike_server_s *S, Lock &lk, int64_t bytes, std::vector<spike_handle> &victims) {
  if (bytes > S->cfg.budget_bytes) return false;
  while (S->used + bytes > S->cfg.budget_bytes) {
    Fac *v = nullptr;
    for (auto &kv : S->mats)
      for (auto &f : kv.second.fac)
        if (f.resident && !f.busy && (!v || evict_before(S, f, *v))) v = &f;
    if (v) {
      if (S->policy == SPIKE_SERVE_EVICT_COST) S->gd_L = std::max(S->gd_L, v->prio);
      victims.push_back(v->h);
      account(S, -v->bytes);
      v->h = nullptr;
      v->bytes = 0;
      v->resident = false;
      ++S->nevict;
      continue;
    }
    if (S->running - S->waiting <= 1) return false;  // nobody else will release anything
    ++S->nwait;
    ++S->waiting;
    S->cv_done.wait(lk);
    --S->waiting;
  }
  account(S, bytes);
  return true;
}

// Take the oldest waiting request whose factorization is not in use, and every other
// waiting request with the same key, up to max_batch_rhs columns (the first is always
// taken).  Returns false when nothing can run now.
bool pick(spike_server_s *S, std::vector<int64_t> &batch) {
  batch.clear();
  size_t first = S->pending.size();
  for (size_t i = 0; i < S->pending.size(); ++i) {
    const Req &r = S->reqs[S->pending[i]];
    if (!S->mats[r.mid].fac[r.prec].busy) {
      first = i;
      break;
    }
  }
  if (first == S->pending.size()) return false;
  const Req &r0 = S->reqs[S->pending[first]];
  int cols = 0;
  std::deque<int64_t> rest;
  for (size_t i = 0; i < S->pending.size(); ++i) {
    const int64_t id = S->pending[i];
    const Req &r = S->reqs[id];
    const bool same = i >= first && r.mid == r0.mid && r.prec == r0.prec && r.trans == r0.trans;
    if (same && (batch.empty() || cols + r.nrhs <= S->cfg.max_batch_rhs)) {
      batch.push_back(id);
      cols += r.nrhs;
    } else {
      rest.push_back(id);
    }
  }
  S->pending.swap(rest);
  return true;
}

// Free evicted factorizations outside the lock (spike_free waits for the stream).
void release(Lock &lk, std::vector<spike_handle> &victims, cudaStream_t st) {
  if (victims.empty()) return;
  lk.unlock();
  for (auto h : victims) {
    if (!h) continue;
    spike_set_stream(h, st);
    spike_free(h);
  }
  victims.clear();
  lk.lock();
}

// Requests of one matrix merged into a solve.
struct Group {
  Mat *M;
  Fac *F;
  std::vector<int64_t> ids;
  int cols;
};

// Add up to `limit` more groups to a solve: waiting FP64 requests with the given trans on
// other matrices whose (non-pivoting) factorization is resident and idle, each with the
// other waiting requests on its matrix, up to max_batch_rhs columns per matrix.
void pick_more(spike_server_s *S, char trans, int64_t mid0, int limit, std::vector<Group> &out) {
  std::unordered_map<int64_t, size_t> gi;
  std::deque<int64_t> rest;
  for (int64_t id : S->pending) {
    const Req &r = S->reqs[id];
    bool take = false;
    if (r.prec == 0 && r.trans == trans && r.mid != mid0) {
      Mat &M = S->mats[r.mid];
      auto it = gi.find(r.mid);
      if (it != gi.end()) {
        Group &g = out[it->second];
        if (g.cols + r.nrhs <= S->cfg.max_batch_rhs) {
          g.ids.push_back(id);
          g.cols += r.nrhs;
          take = true;
        }
      } else if ((int)gi.size() < limit && !M.pivot && M.fac[0].resident && !M.fac[0].busy) {
        gi[r.mid] = out.size();
        out.push_back(Group{&M, &M.fac[0], {id}, r.nrhs});
        M.fac[0].busy = true;
        take = true;
      }
    }
    if (!take) rest.push_back(id);
  }
  S->pending.swap(rest);
}

int grow(spike_server_s *S, Lock &lk, char **p, int64_t *have, int64_t need, cudaStream_t st) {
  if (need <= *have) return 0;
  std::vector<spike_handle> victims;
  const bool ok = admit(S, lk, need - *have, victims);
  release(lk, victims, st);
  if (!ok) return SPIKE_ENOMEM;
  lk.unlock();
  int rc = 0;
  if (!S->dry) {
    if (*p) cudaFreeAsync(*p, st);
    *p = nullptr;
    if (spk::dev_alloc((void **)p, (size_t)need, st) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      rc = SPIKE_ENOMEM;
    }
  }
  lk.lock();
  if (rc) {
    account(S, -*have - (need - *have));
    *have = 0;
    return rc;
  }
  *have = need;
  return 0;
}

void worker(spike_server_s *S, int w) {
  if (!S->dry) cudaSetDevice(S->dev);
  cudaStream_t st = S->dry ? nullptr : S->st[w];
  WorkerBuf &B = S->wb[w];
  Lock lk(S->mu);
  std::vector<int64_t> batch;
  for (;;) {
    while (!pick(S, batch)) {
      if (S->stop && S->pending.empty()) return;
      S->cv_work.wait(lk);
    }
    ++S->running;
    const Req &r0 = S->reqs[batch[0]];
    Mat &M = S->mats[r0.mid];
    const int prec = r0.prec;
    const char trans = r0.trans;
    Fac &F = M.fac[prec];
    F.busy = true;
    int cols = 0;
    for (int64_t id : batch) cols += S->reqs[id].nrhs;
    int rc = 0;

    // 1. factorization on first use (or after eviction)
    if (!F.resident) {
      spike_options o;
      memset(&o, 0, sizeof(o));
      o.K = S->cfg.K;
      o.nrhs_hint = S->cfg.nrhs_hint > 0 ? S->cfg.nrhs_hint : 16;
      o.flags = SPIKE_FLAG_STAGE_BALANCE | SPIKE_FLAG_BATCH_INVARIANT | (prec ? SPIKE_FLAG_MIXED : 0) |
                ((prec && (S->cfg.flags & SPIKE_SERVE_FP64_RESIDUAL)) ? SPIKE_FLAG_FP64_RESIDUAL : 0) |
                (M.host ? 0 : SPIKE_FLAG_BORROW_BAND) |
                ((S->cfg.flags & SPIKE_SERVE_GRAPHS) && !prec ? SPIKE_FLAG_GRAPHS : 0);
      // SPIKE_SERVE_TUNED: the size class's measured worker count, or tune it now
      bool tune_now = false;
      std::pair<int, int> cls(0, std::max(M.kl, M.ku));
      if ((S->cfg.flags & SPIKE_SERVE_TUNED) && S->cfg.p == 0 && !M.host && !S->dry && !M.pivot) {
        while ((2LL << cls.first) <= M.n) ++cls.first;
        auto it = S->tuned.find(cls);
        if (it != S->tuned.end()) {
          M.p = it->second;
        } else if (!S->tuning.count(cls)) {
          S->tuning.insert(cls);
          tune_now = true;
        }
      }
      o.stream = st;
      int64_t res = 0, tr = 0;
      rc = spike_factor_bytes(M.n, M.kl, M.ku, M.p, M.pivot, &o, M.host ? 1 : 0, &res, &tr);
      const int64_t slack = 1 << 20;  // descriptor buffer
      const int64_t reserve = res + tr + slack;
      std::vector<spike_handle> victims;
      if (rc == 0 && !admit(S, lk, reserve, victims)) rc = SPIKE_ENOMEM;
      release(lk, victims, st);
      if (rc == 0) {
        F.bytes = reserve;
        lk.unlock();
        spike_handle h = nullptr;
        int64_t actual = res + slack;
        if (tune_now) {
          // a few worker counts around the rule, factor + one solve of nrhs_hint columns each
          const int64_t kk = std::max(1, std::max(M.kl, M.ku));
          const int pmax = (int)std::max<int64_t>(1, M.n / (4 * kk));
          std::vector<int> cand;
          for (int c : {std::max(1, M.p / 2), M.p, 2 * M.p, 4 * M.p})
            if (c <= pmax && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
          spike_tune_result tr_;
          const int trc = spike_tune(M.band, M.ldab, M.n, M.kl, M.ku, o.nrhs_hint, 1, cand.data(), (int)cand.size(),
                                     nullptr, 0, st, nullptr, &tr_);
          lk.lock();
          if (trc == 0) {
            S->tuned[cls] = tr_.best_p;
            M.p = tr_.best_p;
          }
          S->tuning.erase(cls);
          lk.unlock();
        }
        const double t_fac = now_s();
        if (S->dry) {
          sleep_us(S->cfg.dryrun_factor_us);
        } else {
          rc = spike_factor_ex(M.band, M.ldab, M.n, M.kl, M.ku, M.p, M.pivot, &o, &h);
          if (h) {
            spike_info info;
            if (spike_get_info(h, &info) == 0) actual = info.device_bytes;
          }
          if (rc < 0 && h) {
            spike_free(h);
            h = nullptr;
          }
        }
        const double fac_s = now_s() - t_fac;
        lk.lock();
        ++S->nfact;
        if (rc >= 0) {  // rc > 0: singular (pivoting); kept, its solves report rc
          account(S, actual - F.bytes);
          F.bytes = actual;
          F.h = h;
          F.resident = true;
          F.cost_s = std::max(fac_s, 1e-6);
          F.uses = 0;
        } else {
          account(S, -F.bytes);
          F.bytes = 0;
        }
      }
    }

    // 2. other resident FP64 matrices with waiting requests of the same trans join the
    // solve (one spike_solve_batch: every stage of all of them in shared launches)
    std::vector<Group> groups;
    groups.push_back(Group{&M, &F, batch, cols});
    if (rc == 0 && prec == 0 && !M.pivot && S->batch_systems > 1)
      pick_more(S, trans, r0.mid, S->batch_systems - 1, groups);
    const bool multi = groups.size() > 1;
    // SPIKE_SERVE_GRAPHS: a single-matrix FP64 solve runs as the next power of two of columns
    const bool graphs = (S->cfg.flags & SPIKE_SERVE_GRAPHS) && !multi && prec == 0 && !S->dry;
    int scols = cols;
    if (graphs)
      while (scols & (scols - 1)) scols += scols & -scols;  // round up to a power of two
    if (graphs) groups[0].cols = scols;

    // 3. buffers: merged right-hand sides and solve workspace of this worker
    std::vector<int64_t> fb_off(groups.size(), 0);
    int64_t fb_need = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
      fb_off[g] = fb_need;
      fb_need += ((int64_t)sizeof(double) * groups[g].M->n * groups[g].cols + 255) & ~int64_t(255);
    }
    std::vector<spike_handle> hs;
    std::vector<int> gcols;
    for (auto &g : groups) {
      hs.push_back(g.F->h);
      gcols.push_back(g.cols);
    }
    if (rc == 0) {
      int64_t ws_need = 0;
      if (S->dry) {
        ws_need = 2 * fb_need;
      } else if (multi) {
        rc = spike_solve_batch_workspace(hs.data(), gcols.data(), (int)hs.size(), trans, &ws_need);
      } else {
        rc = spike_solve_workspace(F.h, scols, trans, 0, &ws_need);
      }
      if (rc == 0) rc = grow(S, lk, &B.ws, &B.ws_bytes, ws_need, st);
      if (rc == 0) rc = grow(S, lk, (char **)&B.fb, &B.fb_bytes, fb_need, st);
    }

    // 4. the merged solve
    if (rc == 0) {
      std::vector<std::vector<Req *>> rs(groups.size());
      for (size_t g = 0; g < groups.size(); ++g)
        for (int64_t id : groups[g].ids) rs[g].push_back(&S->reqs[id]);
      lk.unlock();
      if (S->dry) {
        sleep_us(S->cfg.dryrun_solve_us);
        for (size_t g = 0; g < groups.size(); ++g)
          for (Req *r : rs[g]) memmove(r->X, r->F, sizeof(double) * (size_t)groups[g].M->n * r->nrhs);
      } else {
        std::vector<double *> fptr(groups.size());
        for (size_t g = 0; g < groups.size(); ++g) {
          const int64_t n = groups[g].M->n;
          double *base = (double *)((char *)B.fb + fb_off[g]);
          fptr[g] = base;
          int64_t off = 0;
          for (Req *r : rs[g]) {
            if (!rc && cudaMemcpyAsync(base + off * n, r->F, sizeof(double) * n * r->nrhs, cudaMemcpyDefault, st) !=
                           cudaSuccess)
              rc = SPIKE_ECUDA;
            off += r->nrhs;
          }
        }
        if (!rc && scols > cols &&
            cudaMemsetAsync(fptr[0] + (int64_t)cols * M.n, 0, sizeof(double) * M.n * (scols - cols), st) != cudaSuccess)
          rc = SPIKE_ECUDA;
        int64_t replays0 = 0;
        if (graphs && F.h) {
          spike_info gi;
          if (spike_get_info(F.h, &gi) == 0) replays0 = gi.graph_replays;
        }
        if (!rc && multi) {
          rc = spike_solve_batch(hs.data(), fptr.data(), gcols.data(), (int)hs.size(), trans, st, B.ws, B.ws_bytes);
        } else if (!rc) {
          rc = spike_set_stream(F.h, st);
          if (!rc) rc = spike_solve_ws(F.h, fptr[0], M.n, scols, trans, B.ws, B.ws_bytes);
        }
        if (graphs && F.h && !rc) {
          spike_info gi;
          if (spike_get_info(F.h, &gi) == 0) {
            lk.lock();
            S->greplays += gi.graph_replays - replays0;
            lk.unlock();
          }
        }
        for (size_t g = 0; g < groups.size(); ++g) {
          const int64_t n = groups[g].M->n;
          int64_t off = 0;
          for (Req *r : rs[g]) {
            if (!rc && cudaMemcpyAsync(r->X, fptr[g] + off * n, sizeof(double) * n * r->nrhs, cudaMemcpyDefault, st) !=
                           cudaSuccess)
              rc = SPIKE_ECUDA;
            off += r->nrhs;
          }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = SPIKE_ECUDA;
      }
      lk.lock();
      if (!S->dry && !multi && F.h) {
        spike_info info;  // the descriptor buffer may have grown
        if (spike_get_info(F.h, &info) == 0) {
          account(S, info.device_bytes - F.bytes);
          F.bytes = info.device_bytes;
        }
      }
    }

    // 5. completion
    if (rc != 0) {
      const char *msg = spike_last_cuda_error();
      S->last_error = std::string(spike_strerror(rc)) + (msg && *msg ? std::string(": ") + msg : std::string());
    }
    const double t = now_s();
    int nreq = 0;
    for (auto &g : groups) {
      for (int64_t id : g.ids) {
        Req &r = S->reqs[id];
        r.status = rc;
        r.t_done = t;
        r.done = true;
        S->lat.push_back(1e3 * (t - r.t_submit));
        if (rc == 0) ++S->completed;
        else ++S->failed;
      }
      nreq += (int)g.ids.size();
      S->rhs += g.cols;
      g.F->last_use = ++S->tick;
      g.F->busy = false;
      ++g.F->uses;
      g.F->prio = S->gd_L + (double)g.F->uses * g.F->cost_s / (double)std::max<int64_t>(g.F->bytes, 1);
    }
    ++S->batches;
    if (multi) ++S->multi;
    S->max_batch = std::max(S->max_batch, nreq);
    S->max_systems = std::max(S->max_systems, (int)groups.size());
    S->t_last = t;
    --S->running;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" int spike_server_create(const spike_server_config *cfg, spike_server *out) {
  if (!out) return -2;
  *out = nullptr;
  if (!cfg || cfg->budget_bytes <= 0 || cfg->streams < 1 || cfg->streams > 64 || cfg->max_batch_rhs < 1 ||
      cfg->p < 0 || (cfg->evict_policy != SPIKE_SERVE_EVICT_LRU && cfg->evict_policy != SPIKE_SERVE_EVICT_COST))
    return -1;
  spike_server_s *S = new spike_server_s();
  S->cfg = *cfg;
  S->dry = (cfg->flags & SPIKE_SERVE_DRYRUN) != 0;
  if (cfg->batch_systems > 0) S->batch_systems = cfg->batch_systems;
  S->policy = cfg->evict_policy;
  if (!S->dry) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      delete S;
      return SPIKE_ENOGPU;
    }
    cudaGetDevice(&S->dev);
    if (cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->dev) != cudaSuccess) {
      cudaGetLastError();
      S->sms = 152;
    }
    S->st.resize(cfg->streams);
    for (auto &s : S->st)
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s = nullptr;
        spike_server_destroy(S);
        return SPIKE_ECUDA;
      }
  }
  S->wb.resize(cfg->streams);
  for (int w = 0; w < cfg->streams; ++w) S->th.emplace_back(worker, S, w);
  *out = S;
  return 0;
}

extern "C" int spike_server_add_matrix(spike_server S, int64_t id, const double *band, int64_t ldab, int64_t n,
                                       int kl, int ku, int pivot) {
  if (!S) return -1;
  if (!band) return -3;
  if (n < 1) return -5;
  if (kl < 0 || (n > 1 && kl >= n)) return -6;
  if (ku < 0 || (n > 1 && ku >= n)) return -7;
  if (ldab < (int64_t)kl + ku + 1) return -4;
  if (pivot != 0 && pivot != 1) return -8;
  if (std::max(kl, ku) > SPIKE_MAX_K) return SPIKE_ENOTSUP;
  Mat M;
  M.band = band;
  M.ldab = ldab;
  M.n = n;
  M.kl = kl;
  M.ku = ku;
  M.pivot = pivot;
  // Default worker count: blocks of at least 16k rows, and no more blocks than about two
  // per SM for each stream (concurrent requests share the GPU).  Fewer blocks also mean
  // fewer merge levels, whose spike tips (4k^2 per block per level) dominate the
  // footprint of small-n/k factorizations.
  const int64_t k = std::max(1, std::max(kl, ku));
  const int64_t cap = std::max<int64_t>(4, 2 * (int64_t)S->sms / S->cfg.streams);
  M.p = S->cfg.p > 0 ? S->cfg.p : (int)std::min<int64_t>(cap, std::max<int64_t>(1, n / (16 * k)));
  if (S->dry) {
    M.host = true;
  } else {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, band) != cudaSuccess) {
      cudaGetLastError();
      M.host = true;
    } else {
      M.host = !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    }
  }
  Lock lk(S->mu);
  if (S->mats.count(id)) return -2;
  S->mats.emplace(id, M);
  return 0;
}

extern "C" int64_t spike_server_submit(spike_server S, int64_t matrix_id, const double *F, double *X, int nrhs,
                                       char trans, int precision) {
  if (!S) return -1;
  if (!F) return -3;
  if (!X) return -4;
  if (nrhs < 1) return -5;
  if (trans == 'n') trans = 'N';
  if (trans == 't' || trans == 'C' || trans == 'c') trans = 'T';
  if (trans != 'N' && trans != 'T') return -6;
  if (precision != 0 && precision != 1) return -7;
  Lock lk(S->mu);
  auto it = S->mats.find(matrix_id);
  if (it == S->mats.end()) return -2;
  if (precision == 1 && it->second.pivot) return SPIKE_ENOTSUP;
  Req r;
  r.mid = matrix_id;
  r.F = F;
  r.X = X;
  r.nrhs = nrhs;
  r.trans = trans;
  r.prec = precision;
  r.t_submit = now_s();
  if (S->t_first < 0) S->t_first = r.t_submit;
  const int64_t id = (int64_t)S->reqs.size();
  S->reqs.push_back(r);
  S->pending.push_back(id);
  S->cv_work.notify_one();
  return id;
}

extern "C" int spike_server_wait(spike_server S, int64_t req, double *latency_ms) {
  if (!S) return -1;
  Lock lk(S->mu);
  if (req < 0 || req >= (int64_t)S->reqs.size()) return -2;
  S->cv_done.wait(lk, [&] { return S->reqs[req].done; });
  const Req &r = S->reqs[req];
  if (latency_ms) *latency_ms = 1e3 * (r.t_done - r.t_submit);
  return r.status;
}

extern "C" int spike_server_request_latency(spike_server S, int64_t req, double *latency_ms) {
  if (!S) return -1;
  Lock lk(S->mu);
  if (req < 0 || req >= (int64_t)S->reqs.size()) return -2;
  const Req &r = S->reqs[req];
  if (!r.done) return 1;
  if (latency_ms) *latency_ms = 1e3 * (r.t_done - r.t_submit);
  return 0;
}

extern "C" int spike_server_drain(spike_server S) {
  if (!S) return -1;
  Lock lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->completed + S->failed == (int64_t)S->reqs.size(); });
  return 0;
}

extern "C" int spike_server_stats_get(spike_server S, spike_server_stats *o) {
  if (!S) return -1;
  if (!o) return -2;
  Lock lk(S->mu);
  memset(o, 0, sizeof(*o));
  o->submitted = (int64_t)S->reqs.size();
  o->completed = S->completed;
  o->failed = S->failed;
  o->batches = S->batches;
  o->rhs = S->rhs;
  o->factorizations = S->nfact;
  o->evictions = S->nevict;
  o->admission_waits = S->nwait;
  o->used_bytes = S->used;
  o->peak_bytes = S->peak;
  for (auto &kv : S->mats)
    for (auto &f : kv.second.fac) o->resident += f.resident ? 1 : 0;
  o->max_batch = S->max_batch;
  o->multi_solves = S->multi;
  o->max_systems = S->max_systems;
  o->tuned_classes = (int32_t)S->tuned.size();
  o->graph_replays = S->greplays;
  if (!S->lat.empty()) {
    std::vector<double> v = S->lat;
    std::sort(v.begin(), v.end());
    auto rank = [&](double q) {  // nearest-rank percentile
      size_t i = (size_t)std::ceil(q * (double)v.size());
      return v[std::min(v.size(), std::max<size_t>(i, 1)) - 1];
    };
    o->p50_ms = rank(0.50);
    o->p99_ms = rank(0.99);
    o->max_ms = v.back();
    double s = 0.0;
    for (double x : v) s += x;
    o->mean_ms = s / (double)v.size();
    o->span_s = S->t_last - S->t_first;
    if (o->span_s > 0) {
      o->solves_per_s = (double)S->completed / o->span_s;
      o->rhs_per_s = (double)S->rhs / o->span_s;
    }
  }
  return 0;
}

extern "C" int spike_server_latencies(spike_server S, double *ms, int64_t cap, int64_t *count) {
  if (!S) return -1;
  Lock lk(S->mu);
  const int64_t n = (int64_t)S->lat.size();
  if (count) *count = n;
  if (ms)
    for (int64_t i = 0; i < std::min(cap, n); ++i) ms[i] = S->lat[i];
  return 0;
}

extern "C" const char *spike_server_last_error(spike_server S) {
  if (!S) return "";
  Lock lk(S->mu);
  thread_local std::string copy;
  copy = S->last_error;
  return copy.c_str();
}

extern "C" void spike_server_destroy(spike_server S) {
  if (!S) return;
  {
    Lock lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto &t : S->th)
    if (t.joinable()) t.join();
  if (!S->dry) {
    cudaSetDevice(S->dev);
    for (auto &kv : S->mats)
      for (auto &f : kv.second.fac)
        if (f.h) spike_free(f.h);
    for (size_t w = 0; w < S->wb.size(); ++w) {
      cudaStream_t s = w < S->st.size() ? S->st[w] : nullptr;
      if (S->wb[w].ws) cudaFreeAsync(S->wb[w].ws, s);
      if (S->wb[w].fb) cudaFreeAsync(S->wb[w].fb, s);
    }
    for (auto &s : S->st)
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
  }
  delete S;
}
