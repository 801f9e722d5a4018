// Batched runtime behind the C ABI: many independent noisy circuits ("instances") on one GPU.
//
// Instances whose gates sit on the same positions in the same order (same qubit count, same
// sequence of (1q/2q, site)) form a group.  A group runs as one or more handles of the engine, each
// a batch of chains that every call advances at once, each chain with its own gate matrices and
// channels (device arrays, uploaded once).  Each handle's whole circuit, reset included, is captured
// into one CUDA graph on its own stream, so a run replays every graph without host work in between
// and the groups' launches overlap on the GPU.
//
// The schedule of a group (how many handles its chains are split over, and whether the complex64
// products use the tensor cores) is chosen by a small autotuner: every candidate is built, captured
// and timed over two replays with CUDA events, and the fastest is kept.  Results are persisted in a
// JSON file keyed by the group's shape, so later runs with the same file take the stored choice
// without timing.  Groups smaller than kTuneMinChains use the default schedule (one handle, tensor
// cores on in the complex64 modes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "bounds.cuh"
#include "mpdo.h"

namespace {

constexpr int kTuneMinChains = 128;

struct BatchHandle {
  mpdo_t h = nullptr;
  cudaStream_t stream = nullptr;
  mpdo_graph_t graph = nullptr;
  std::vector<int> inst;           // instance of each chain
  std::vector<mpdo_chan_t> chans;  // one channel set per distinct set of process matrices
  std::vector<void*> dev;          // gate matrices and channel index arrays (device)
  void release() {
    if (graph) mpdo_graph_free(graph);
    for (mpdo_chan_t c : chans) channel_free(c);
    if (h) mpdo_free(h);
    for (void* p : dev) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
    graph = nullptr;
    chans.clear();
    dev.clear();
    h = nullptr;
    stream = nullptr;
  }
};

struct BatchGroup {
  int n = 0;
  std::vector<int> inst;        // instances of the group
  int first_op_instance = 0;    // an instance whose op list defines the signature
  int handles = 1, tensor_cores = 1;
  double tuned_ms = 0;
  std::vector<BatchHandle> hs;
};

struct Program {  // the caller's arrays, copied
  int count = 0;
  std::vector<int> n, op_begin, op_kind, op_q, op_chi, chi_nq, chi_off;
  std::vector<double> op_U, chis;
};

}  // namespace

struct mpdo_batch {
  Program prog;
  int chi_max = 1, kappa_max = 1, prec = 0;
  std::vector<BatchGroup> groups;
  long long n2q = 0;
};

namespace {

mpdo_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MPDO_OK : MPDO_ECUDA; }

// One handle over the instances `inst` of a group, with its circuit captured into a graph.
mpdo_status build_handle(const Program& P, const BatchGroup& g, const std::vector<int>& inst, int chi_max,
                         int kappa_max, int prec, int tc, BatchHandle& out) {
  BatchHandle H;
  H.inst = inst;
  const int B = (int)inst.size();
  mpdo_status st = cuda_status(cudaStreamCreateWithFlags(&H.stream, cudaStreamNonBlocking));
  if (!st) st = mpdo_init_batch(B, g.n, chi_max, kappa_max, prec, (void*)H.stream, &H.h);
  if (!st && prec != MPDO_FP64) st = mpdo_set_tensor_cores(H.h, tc);
  const int c0 = g.first_op_instance;
  const int nops = P.op_begin[c0 + 1] - P.op_begin[c0];
  std::map<std::vector<int>, mpdo_chan_t> cache;  // distinct chi index lists -> channel set
  struct Slot {
    int kind, q;
    double* U;
    mpdo_chan_t ch;
    int* idx;
  };
  std::vector<Slot> slots;
  for (int k = 0; k < nops && !st; ++k) {
    const int o0 = P.op_begin[c0] + k;
    const int kind = P.op_kind[o0], q = P.op_q[o0], d = 1 << kind;
    if (kind == MPDO_OP_TRUNCATE_BONDS) {
      slots.push_back({kind, q, nullptr, nullptr, nullptr});
      continue;
    }
    // gate matrices of every chain, row-major d x d complex
    std::vector<double> U((size_t)B * 2 * d * d);
    std::vector<int> chi_of(B);
    for (int b = 0; b < B; ++b) {
      const int o = P.op_begin[inst[b]] + k;
      std::memcpy(&U[(size_t)b * 2 * d * d], &P.op_U[(size_t)o * 32], sizeof(double) * 2 * d * d);
      chi_of[b] = P.op_chi[o];
    }
    // distinct process matrices of this position, and each chain's index into them
    std::vector<int> uniq(chi_of);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    std::vector<int> idx(B);
    for (int b = 0; b < B; ++b) idx[b] = (int)(std::lower_bound(uniq.begin(), uniq.end(), chi_of[b]) - uniq.begin());
    mpdo_chan_t ch = nullptr;
    auto it = cache.find(uniq);
    if (it != cache.end()) {
      ch = it->second;
    } else {
      const int d2 = d * d;
      std::vector<double> chis((size_t)uniq.size() * 2 * d2 * d2);
      for (size_t u = 0; u < uniq.size(); ++u) {
        if (P.chi_nq[uniq[u]] != kind) {
          st = MPDO_EINVAL;
          break;
        }
        std::memcpy(&chis[u * 2 * d2 * d2], &P.chis[P.chi_off[uniq[u]]], sizeof(double) * 2 * d2 * d2);
      }
      if (!st) st = channel_set_from_process_matrices(H.h, kind, (int)uniq.size(), chis.data(), 0.0, &ch, nullptr);
      if (st) break;
      cache[uniq] = ch;
      H.chans.push_back(ch);
    }
    double* Ud = nullptr;
    int* idd = nullptr;
    st = cuda_status(cudaMalloc((void**)&Ud, sizeof(double) * U.size()));
    if (!st) H.dev.push_back(Ud);
    if (!st) st = cuda_status(cudaMalloc((void**)&idd, sizeof(int) * B));
    if (!st) H.dev.push_back(idd);
    if (!st) st = cuda_status(cudaMemcpy(Ud, U.data(), sizeof(double) * U.size(), cudaMemcpyHostToDevice));
    if (!st) st = cuda_status(cudaMemcpy(idd, idx.data(), sizeof(int) * B, cudaMemcpyHostToDevice));
    slots.push_back({kind, q, Ud, ch, idd});
  }
  if (!st) st = mpdo_capture_begin(H.h);
  if (!st) {
    mpdo_status cs = mpdo_reset(H.h);
    for (const Slot& s : slots) {
      if (cs) break;
      cs = s.kind == 1   ? apply_1q_batch(H.h, s.q, s.U, s.ch, s.idx)
           : s.kind == 2 ? apply_2q_batch(H.h, s.q, s.U, s.ch, s.idx)
                         : truncate_bonds(H.h, s.q, nullptr);
    }
    mpdo_status es = mpdo_capture_end(H.h, 0, &H.graph);
    st = cs ? cs : es;
  }
  if (st) {
    H.release();
    return st;
  }
  out = H;
  return MPDO_OK;
}

mpdo_status build_group(const Program& P, BatchGroup& g, int chi_max, int kappa_max, int prec) {
  const int B = (int)g.inst.size();
  const int parts = std::max(1, std::min(g.handles, B));
  for (int s = 0; s < parts; ++s) {
    const int b0 = (int)((long long)B * s / parts), b1 = (int)((long long)B * (s + 1) / parts);
    std::vector<int> sub(g.inst.begin() + b0, g.inst.begin() + b1);
    BatchHandle H;
    mpdo_status st = build_handle(P, g, sub, chi_max, kappa_max, prec, g.tensor_cores, H);
    if (st) return st;
    g.hs.push_back(H);
  }
  return MPDO_OK;
}

void release_group(BatchGroup& g) {
  for (auto& H : g.hs) H.release();
  g.hs.clear();
}

// Time two replays of the group's graphs (all handles concurrently), milliseconds per replay.
mpdo_status time_group(BatchGroup& g, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s0 = g.hs[0].stream;
  mpdo_status st = cuda_status(cudaEventCreate(&e0));
  if (!st) st = cuda_status(cudaEventCreate(&e1));
  for (auto& H : g.hs)
    if (!st) st = mpdo_graph_launch(H.graph);  // warm-up
  if (!st) st = cuda_status(cudaDeviceSynchronize());
  if (!st) st = cuda_status(cudaEventRecord(e0, s0));
  for (auto& H : g.hs)
    if (!st && H.stream != s0) st = cuda_status(cudaStreamWaitEvent(H.stream, e0, 0));
  for (int r = 0; r < 2 && !st; ++r)
    for (auto& H : g.hs)
      if (!st) st = mpdo_graph_launch(H.graph);
  std::vector<cudaEvent_t> ends;
  for (auto& H : g.hs) {
    if (st || H.stream == s0) continue;
    cudaEvent_t d = nullptr;
    st = cuda_status(cudaEventCreateWithFlags(&d, cudaEventDisableTiming));
    if (!st) ends.push_back(d);
    if (!st) st = cuda_status(cudaEventRecord(d, H.stream));
    if (!st) st = cuda_status(cudaStreamWaitEvent(s0, d, 0));
  }
  if (!st) st = cuda_status(cudaEventRecord(e1, s0));
  if (!st) st = cuda_status(cudaEventSynchronize(e1));
  float t = 0;
  if (!st) st = cuda_status(cudaEventElapsedTime(&t, e0, e1));
  if (!st) *ms = t / 2.0;
  for (cudaEvent_t d : ends) cudaEventDestroy(d);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

// ---- the tuning file: {"entries": [{"key": "...", "handles": h, "tensor_cores": t, "ms": m}, ...]}
struct TuneEntry {
  int handles, tensor_cores;
  double ms;
};

std::map<std::string, TuneEntry> read_tuning(const char* path) {
  std::map<std::string, TuneEntry> out;
  if (!path) return out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  size_t pos = 0;
  while ((pos = text.find("\"key\": \"", pos)) != std::string::npos) {
    pos += 8;
    const size_t end = text.find('"', pos);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos, end - pos);
    TuneEntry e{1, 1, 0.0};
    const size_t obj_end = text.find('}', end);
    const std::string obj = text.substr(end, obj_end == std::string::npos ? std::string::npos : obj_end - end);
    const size_t ph = obj.find("\"handles\": "), pt = obj.find("\"tensor_cores\": "), pm = obj.find("\"ms\": ");
    if (ph != std::string::npos) e.handles = std::atoi(obj.c_str() + ph + 11);
    if (pt != std::string::npos) e.tensor_cores = std::atoi(obj.c_str() + pt + 16);
    if (pm != std::string::npos) e.ms = std::atof(obj.c_str() + pm + 6);
    if (e.handles >= 1) out[key] = e;
    pos = end;
  }
  return out;
}

bool write_tuning(const char* path, const std::map<std::string, TuneEntry>& entries) {
  FILE* f = std::fopen(path, "wb");
  if (!f) return false;
  std::fprintf(f, "{\"entries\": [\n");
  size_t i = 0;
  for (auto& kv : entries) {
    std::fprintf(f, "  {\"key\": \"%s\", \"handles\": %d, \"tensor_cores\": %d, \"ms\": %.4f}%s\n", kv.first.c_str(),
                 kv.second.handles, kv.second.tensor_cores, kv.second.ms, ++i < entries.size() ? "," : "");
  }
  std::fprintf(f, "]}\n");
  return std::fclose(f) == 0;
}

std::string group_key(const Program& P, const BatchGroup& g, int chi_max, int kappa_max, int prec) {
  const int c0 = g.first_op_instance;
  int n1 = 0, n2 = 0, n3 = 0;
  for (int o = P.op_begin[c0]; o < P.op_begin[c0 + 1]; ++o) {
    const int k = P.op_kind[o];
    (k == 1 ? n1 : k == 2 ? n2 : n3)++;
  }
  char buf[192];
  std::snprintf(buf, sizeof(buf), "n=%d ops1=%d ops2=%d sweeps=%d chi=%d kappa=%d prec=%d chains=%d", g.n, n1, n2, n3,
                chi_max, kappa_max, prec, (int)g.inst.size());
  return buf;
}

}  // namespace

extern "C" {

mpdo_status mpdo_batch_create(int count, const int* n_qubits, const int* op_begin, const int* op_kind, const int* op_q,
                              const double* op_U, const int* op_chi, int n_chi, const int* chi_nq, const double* chis,
                              int chi_max, int kappa_max, int prec, const char* tuning_path, mpdo_batch_t* out) {
  if (count < 1 || !n_qubits || !op_begin || !op_kind || !op_q || !op_U || !op_chi || n_chi < 1 || !chi_nq || !chis ||
      !out)
    return MPDO_EINVAL;
  if (prec != MPDO_FP64 && prec != MPDO_MIXED && prec != MPDO_FP32) return MPDO_EINVAL;
  std::unique_ptr<mpdo_batch> b(new (std::nothrow) mpdo_batch());
  if (!b) return MPDO_ENOMEM;
  Program& P = b->prog;
  P.count = count;
  P.n.assign(n_qubits, n_qubits + count);
  P.op_begin.assign(op_begin, op_begin + count + 1);
  const int nops = op_begin[count];
  if (op_begin[0] != 0 || nops < 0) return MPDO_EINVAL;
  for (int c = 0; c < count; ++c)
    if (op_begin[c + 1] < op_begin[c] || P.n[c] < 1) return MPDO_EINVAL;
  P.op_kind.assign(op_kind, op_kind + nops);
  P.op_q.assign(op_q, op_q + nops);
  P.op_chi.assign(op_chi, op_chi + nops);
  P.op_U.assign(op_U, op_U + (size_t)nops * 32);
  P.chi_nq.assign(chi_nq, chi_nq + n_chi);
  P.chi_off.resize(n_chi);
  size_t off = 0;
  for (int m = 0; m < n_chi; ++m) {
    if (chi_nq[m] != 1 && chi_nq[m] != 2) return MPDO_EINVAL;
    P.chi_off[m] = (int)off;
    const int d2 = 1 << (2 * chi_nq[m]);
    off += (size_t)2 * d2 * d2;
  }
  P.chis.assign(chis, chis + off);
  for (int c = 0; c < count; ++c)
    for (int o = op_begin[c]; o < op_begin[c + 1]; ++o) {
      const int k = P.op_kind[o], q = P.op_q[o];
      if (k == MPDO_OP_TRUNCATE_BONDS) {
        if (q < 1 || q > chi_max) return MPDO_EINVAL;
        continue;
      }
      if ((k != 1 && k != 2) || q < 0 || q + k > P.n[c] || P.op_chi[o] < 0 || P.op_chi[o] >= n_chi ||
          P.chi_nq[P.op_chi[o]] != k)
        return MPDO_EINVAL;
    }
  b->chi_max = chi_max;
  b->kappa_max = kappa_max;
  b->prec = prec;
  // group by signature (n, sequence of (kind, site))
  std::map<std::vector<int>, int> by_sig;
  for (int c = 0; c < count; ++c) {
    std::vector<int> sig{P.n[c]};
    for (int o = op_begin[c]; o < op_begin[c + 1]; ++o) {
      sig.push_back(P.op_kind[o]);
      sig.push_back(P.op_q[o]);
      if (P.op_kind[o] == 2) ++b->n2q;
    }
    auto it = by_sig.find(sig);
    if (it == by_sig.end()) {
      by_sig[sig] = (int)b->groups.size();
      BatchGroup g;
      g.n = P.n[c];
      g.first_op_instance = c;
      g.inst.push_back(c);
      g.tensor_cores = prec != MPDO_FP64 ? 1 : 0;
      b->groups.push_back(g);
    } else {
      b->groups[it->second].inst.push_back(c);
    }
  }
  // schedules: stored, tuned (large groups, when a tuning file is given) or default
  std::map<std::string, TuneEntry> tune = read_tuning(tuning_path);
  bool tuned_any = false;
  for (BatchGroup& g : b->groups) {
    const std::string key = group_key(P, g, chi_max, kappa_max, prec);
    auto it = tune.find(key);
    if (it != tune.end()) {
      g.handles = it->second.handles;
      g.tensor_cores = prec != MPDO_FP64 ? it->second.tensor_cores : 0;
      g.tuned_ms = it->second.ms;
    } else if (tuning_path && (int)g.inst.size() >= kTuneMinChains) {
      double best = 1e300;
      int bh = 1, bt = g.tensor_cores;
      for (int h : {1, 2, 4}) {
        for (int tc : {1, 0}) {
          if (tc == 1 && prec == MPDO_FP64) continue;
          BatchGroup trial = g;
          trial.handles = h;
          trial.tensor_cores = tc;
          double ms = 0;
          mpdo_status st = build_group(P, trial, chi_max, kappa_max, prec);
          if (!st) st = time_group(trial, &ms);
          release_group(trial);
          if (st == MPDO_ENOMEM) continue;
          if (st) {
            for (BatchGroup& gg : b->groups) release_group(gg);
            return st;
          }
          if (ms < best) {
            best = ms;
            bh = h;
            bt = tc;
          }
        }
      }
      g.handles = bh;
      g.tensor_cores = bt;
      g.tuned_ms = best;
      tune[key] = TuneEntry{bh, bt, best};
      tuned_any = true;
    }
    mpdo_status st = build_group(P, g, chi_max, kappa_max, prec);
    if (st) {
      for (BatchGroup& gg : b->groups) release_group(gg);
      return st;
    }
  }
  if (tuned_any && tuning_path && !write_tuning(tuning_path, tune)) {
    for (BatchGroup& gg : b->groups) release_group(gg);
    return MPDO_EINVAL;
  }
  *out = b.release();
  return MPDO_OK;
}

mpdo_status mpdo_batch_run(mpdo_batch_t b) {
  if (!b) return MPDO_EINVAL;
  for (BatchGroup& g : b->groups)
    for (BatchHandle& H : g.hs) {
      mpdo_status st = mpdo_graph_launch(H.graph);
      if (st) return st;
    }
  return MPDO_OK;
}

mpdo_status mpdo_batch_sync(mpdo_batch_t b) {
  if (!b) return MPDO_EINVAL;
  mpdo_status first = MPDO_OK;
  for (BatchGroup& g : b->groups)
    for (BatchHandle& H : g.hs) {
      mpdo_status st = mpdo_sync(H.h);
      if (st && !first) first = st;
    }
  return first;
}

mpdo_status mpdo_batch_expect(mpdo_batch_t b, int kind, const int* arg_begin, const int* args, double* out) {
  if (!b || !out) return MPDO_EINVAL;
  const Program& P = b->prog;
  std::vector<long long> zz_off;
  if (kind == MPDO_EXPECT_ZZ_MAP) {
    zz_off.resize(P.count + 1, 0);
    for (int c = 0; c < P.count; ++c) zz_off[c + 1] = zz_off[c] + (long long)P.n[c] * P.n[c];
  } else if (kind == MPDO_EXPECT_MAXCUT) {
    if (!arg_begin || (!args && arg_begin[P.count] > 0)) return MPDO_EINVAL;
    for (int c = 0; c < P.count; ++c) {
      if (arg_begin[c + 1] < arg_begin[c] || (arg_begin[c + 1] - arg_begin[c]) % 2) return MPDO_EINVAL;
      for (int a = arg_begin[c]; a < arg_begin[c + 1]; ++a)
        if (args[a] < 0 || args[a] >= P.n[c]) return MPDO_EINVAL;
    }
  } else if (kind != MPDO_EXPECT_TRACE && kind != MPDO_EXPECT_GHZ && kind != MPDO_EXPECT_PURITY &&
             kind != MPDO_EXPECT_DISCARDED) {
    return MPDO_EINVAL;
  }
  for (BatchGroup& g : b->groups)
    for (BatchHandle& H : g.hs) {
      const int B = (int)H.inst.size(), n = g.n;
      const int q = kind == MPDO_EXPECT_DISCARDED ? 3 : (kind == MPDO_EXPECT_ZZ_MAP || kind == MPDO_EXPECT_MAXCUT) ? n * n : 1;
      std::vector<double> v((size_t)B * q);
      const int hk = kind == MPDO_EXPECT_MAXCUT ? MPDO_EXPECT_ZZ_MAP : kind;
      mpdo_status st = expect(H.h, hk, nullptr, 0, v.data());
      if (st) return st;
      for (int i = 0; i < B; ++i) {
        const int c = H.inst[i];
        const double* vi = &v[(size_t)i * q];
        if (kind == MPDO_EXPECT_ZZ_MAP) {
          std::memcpy(out + zz_off[c], vi, sizeof(double) * n * n);
        } else if (kind == MPDO_EXPECT_DISCARDED) {
          std::memcpy(out + 3 * (size_t)c, vi, sizeof(double) * 3);
        } else if (kind == MPDO_EXPECT_MAXCUT) {
          double s = 0;
          for (int a = arg_begin[c]; a < arg_begin[c + 1]; a += 2) s += 0.5 * (1.0 - vi[args[a] * n + args[a + 1]]);
          out[c] = s;
        } else {
          out[c] = vi[0];
        }
      }
    }
  return MPDO_OK;
}

mpdo_status mpdo_batch_info(mpdo_batch_t b, int* groups, int* handles, long long* updates_2q) {
  if (!b) return MPDO_EINVAL;
  int nh = 0;
  for (auto& g : b->groups) nh += (int)g.hs.size();
  if (groups) *groups = (int)b->groups.size();
  if (handles) *handles = nh;
  if (updates_2q) *updates_2q = b->n2q;
  return MPDO_OK;
}

mpdo_status mpdo_batch_schedule(mpdo_batch_t b, int group, int* n_qubits, int* chains, int* handles,
                                int* tensor_cores, double* tuned_ms) {
  if (!b || group < 0 || group >= (int)b->groups.size()) return MPDO_EINVAL;
  const BatchGroup& g = b->groups[group];
  if (n_qubits) *n_qubits = g.n;
  if (chains) *chains = (int)g.inst.size();
  if (handles) *handles = (int)g.hs.size();
  if (tensor_cores) *tensor_cores = g.tensor_cores;
  if (tuned_ms) *tuned_ms = g.tuned_ms;
  return MPDO_OK;
}

mpdo_status mpdo_batch_fidelity(mpdo_batch_t a, mpdo_batch_t b, double* out) {
  if (!a || !b || !out || a->prog.count != b->prog.count) return MPDO_EINVAL;
  // (handle, chain) of every instance in each batch
  auto locate = [](mpdo_batch_t x) {
    std::vector<std::pair<mpdo_t, int>> loc(x->prog.count, {nullptr, -1});
    for (BatchGroup& g : x->groups)
      for (BatchHandle& H : g.hs)
        for (size_t i = 0; i < H.inst.size(); ++i) loc[H.inst[i]] = {H.h, (int)i};
    return loc;
  };
  const auto la = locate(a), lb = locate(b);
  for (int c = 0; c < a->prog.count; ++c) {
    if (a->prog.n[c] != b->prog.n[c]) return MPDO_EINVAL;
    mpdo_status st = mpdo_fidelity(la[c].first, la[c].second, lb[c].first, lb[c].second, out + c);
    if (st) return st;
  }
  return MPDO_OK;
}

mpdo_status mpdo_batch_free(mpdo_batch_t b) {
  if (!b) return MPDO_EINVAL;
  for (BatchGroup& g : b->groups) release_group(g);
  delete b;
  return MPDO_OK;
}

}  // extern "C"
