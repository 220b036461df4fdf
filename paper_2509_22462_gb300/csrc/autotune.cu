// Autotuner for the tensor-core GEMMs of a net: for every tangent-GEMM shape it times the N-tile
// widths the kernel supports (over the chain of that shape's layers, as a step runs them), for
// the symmetric product the split-K counts, on the net's own buffers with CUDA events, and keeps
// the fastest.  Results can be kept in a small JSON file
// ({"<key>": [choice, microseconds], ...}, one key per device, kind, precision and shape) so that
// later loads reuse them without timing.
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "net.cuh"

using namespace nnc;

namespace {

std::map<std::string, std::pair<int, double>> read_cache(const char* path) {
  std::map<std::string, std::pair<int, double>> m;
  if (!path) return m;
  std::ifstream f(path);
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  while (true) {
    const size_t k0 = s.find('"', i);
    if (k0 == std::string::npos) break;
    const size_t k1 = s.find('"', k0 + 1);
    const size_t b0 = s.find('[', k1);
    const size_t b1 = s.find(']', b0);
    if (k1 == std::string::npos || b0 == std::string::npos || b1 == std::string::npos) break;
    int choice = 0;
    double us = 0;
    if (std::sscanf(s.c_str() + b0 + 1, "%d , %lf", &choice, &us) == 2)
      m[s.substr(k0 + 1, k1 - k0 - 1)] = {choice, us};
    i = b1 + 1;
  }
  return m;
}

void write_cache(const char* path, const std::map<std::string, std::pair<int, double>>& m) {
  if (!path) return;
  std::ofstream f(path);
  f << "{\n";
  size_t n = 0;
  for (auto& kv : m) {
    f << "  \"" << kv.first << "\": [" << kv.second.first << ", " << kv.second.second << "]";
    f << (++n < m.size() ? ",\n" : "\n");
  }
  f << "}\n";
}

std::string key_of(const nnc_net* net, const char* kind, int M, int N, int K) {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, net->device);
  char b[256];
  std::snprintf(b, sizeof b, "sm%d%d-%dsm %s prec%d M%d N%d K%d", p.major, p.minor,
                p.multiProcessorCount, kind, net->prec, M, N, K);
  return b;
}

// Average microseconds of `reps` runs of fn on st (after one warm-up run).
template <typename F>
double time_us(cudaStream_t st, int reps, F fn) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fn();
  cudaEventRecord(a, st);
  for (int i = 0; i < reps; ++i) fn();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return cudaGetLastError() == cudaSuccess ? 1e3 * ms / reps : 1e30;
}

}  // namespace

extern "C" int nnc_autotune(nnc_net* net, const char* cache_path, int retune) {
  if (!net) {
    set_last_error("net is NULL");
    return NNC_ERR_ARG;
  }
  const int prec = net->prec;
  if (!(prec == NNC_BF16 || prec == NNC_BF16X3 || prec == NNC_FP8)) return NNC_OK;  // CUDA-core forms
  cudaSetDevice(net->device);
  auto cache = read_cache(cache_path);
  cudaStream_t st = net->stream;
  const int n = net->n_in;
  // single-SM N tiles, then SM-pair tiles (negative codes)
  const int bns[8] = {112, 128, 208, 256, -128, -160, -208, -256};
  // tangent GEMMs: layers of one shape share a choice, timed over the chain of those layers as a
  // step runs them (different weights each launch), so that a layer's weights are not timed out
  // of L2, which one repeated launch would do
  std::map<std::string, std::vector<int>> groups;
  for (int l = 1; l < net->L; ++l)
    if (net->layers[l].plan_tan.ready)
      groups[key_of(net, "tangent", net->layers[l].mp, n, net->layers[l].kp)].push_back(l);
  auto make_plan = [&](TcPlan& p, int l, int bn) {
    LayerDev& Ly = net->layers[l];
    const int cur = (l - 1) % 2;
    return prec == NNC_FP8
               ? tc_plan_make(p, TC_TANGENT, prec, Ly.W8, nullptr, Ly.mp, Ly.kp, net->A8, nullptr, n,
                              Ly.kp, Ly.mp, n, Ly.kp, net->sm_count, bn)
               : tc_plan_make(p, TC_TANGENT, prec, Ly.Whi, Ly.Wlo, Ly.mp, Ly.kp, net->At[cur][0],
                              net->At[cur][1], n, Ly.kp, Ly.mp, n, Ly.kp, net->sm_count, bn);
  };
  for (auto& g : groups) {
    const std::vector<int>& ls = g.second;
    int best = plan_code(net->layers[ls[0]].plan_tan);
    auto it = cache.find(g.first);
    if (it != cache.end() && !retune) {
      best = it->second.first;
    } else {
      double best_us = 1e30;
      for (int bn : bns) {
        std::vector<TcPlan> plans(ls.size());
        bool okp = true;
        for (size_t i = 0; i < ls.size() && okp; ++i) okp = make_plan(plans[i], ls[i], bn) == NNC_OK;
        if (!okp) continue;
        // each layer writes its own operand block, as in an evaluation (the first layer's block,
        // written once at load, must stay intact)
        const double us = time_us(st, 3, [&] {
          for (size_t i = 0; i < ls.size(); ++i) {
            LayerDev& Ly = net->layers[ls[i]];
            const int cur = (ls[i] - 1) % 2;
            auto zo = [&](void* base) {
              return (base && Ly.zy_off >= 0) ? (void*)((char*)base + (size_t)Ly.zy_off * 2) : nullptr;
            };
            tc_tangent(plans[i], Ly.s1, Ly.c_f, net->At[1 - cur][0], net->At[1 - cur][1], Ly.mp,
                       zo(net->Zt[0]), zo(net->Zt[1]), zo(net->Yt[0]), zo(net->Yt[1]), net->K_total,
                       net->dev_err, st, Ly.w8s, net->tsc);
          }
        }) / ls.size();
        if (us < best_us) {
          best_us = us;
          best = bn;
        }
      }
      cache[g.first] = {best, best_us};
    }
    // apply the choice through temporaries: a cached entry whose plan fails leaves every layer's
    // current plan in place, is dropped from the cache and reported
    std::vector<TcPlan> fresh(ls.size());
    bool okp = true;
    for (size_t i = 0; i < ls.size() && okp; ++i)
      okp = best == plan_code(net->layers[ls[i]].plan_tan) ||
            make_plan(fresh[i], ls[i], best) == NNC_OK;
    if (!okp) {
      cache.erase(g.first);
      write_cache(cache_path, cache);
      set_last_error("autotune: the tangent tile " + std::to_string(best) + " chosen for " + g.first +
                     " has no valid plan; the previous tiling is kept");
      return NNC_ERR_ARG;
    }
    for (size_t i = 0; i < ls.size(); ++i)
      if (best != plan_code(net->layers[ls[i]].plan_tan)) net->layers[ls[i]].plan_tan = fresh[i];
  }
  // the persistent chain (one launch for every tangent GEMM) against the per-layer launches just
  // chosen, over the same layers and buffers
  if (net->chain_nl > 0) {
    const std::string key = key_of(net, "chain", net->chain_plans[0].M, n, net->chain_nl);
    auto it = cache.find(key);
    int use = 1;
    if (it != cache.end() && !retune) {
      use = it->second.first;
    } else {
      std::vector<ChainOut> outs(net->chain_nl);
      for (int i = 0; i < net->chain_nl; ++i) {
        LayerDev& Ly = net->layers[i + 1];
        const bool last = i + 1 == net->L - 1;
        const int cur = i % 2;
        auto zo = [&](void* base) {
          return (base && Ly.zy_off >= 0) ? (void*)((char*)base + (size_t)Ly.zy_off * 2) : nullptr;
        };
        outs[i] = ChainOut{Ly.s1, Ly.c_f, last ? nullptr : net->At[1 - cur][0],
                           last ? nullptr : net->At[1 - cur][1], Ly.mp, zo(net->Zt[0]), zo(net->Zt[1]),
                           nullptr, nullptr};
      }
      const size_t cb = sizeof(unsigned) * (size_t)net->chain_nl * net->chain_plans[0].ntn;
      const double us_chain = time_us(st, 3, [&] {
        cudaMemsetAsync(net->chain_cnt, 0, cb, st);
        tc_tangent_chain(net->chain_plans.data(), outs.data(), net->chain_nl, net->chain_cnt,
                         net->K_total, net->dev_err, st);
      });
      const double us_layers = time_us(st, 3, [&] {
        for (int i = 0; i < net->chain_nl; ++i) {
          LayerDev& Ly = net->layers[i + 1];
          tc_tangent(Ly.plan_tan, Ly.s1, Ly.c_f, outs[i].at_hi, outs[i].at_lo, Ly.mp, outs[i].zt_hi,
                     outs[i].zt_lo, nullptr, nullptr, net->K_total, net->dev_err, st, Ly.w8s, net->tsc);
        }
      });
      use = us_chain < us_layers ? 1 : 0;
      cache[key] = {use, use ? us_chain : us_layers};
    }
    net->use_chain = use != 0;
  }
  // symmetric product: N tile (128 or 256 columns; lower-triangle tiles only) and split-K count
  // (bounded by the partial-sum buffer allocated at load); the cache keeps bn * 1000 + splits
  if (net->K_total > 0 && net->plan_syrk.ready) {
    const std::string key = key_of(net, "syrk", n, n, net->K_total);
    int best = net->plan_syrk.bn * 1000 + net->plan_syrk.splits;
    auto it = cache.find(key);
    auto valid = [&](int code) {
      return (code / 1000 == 128 || code / 1000 == 256) && code % 1000 >= 1 &&
             code % 1000 <= net->h_splits;
    };
    if (it != cache.end() && !retune && valid(it->second.first)) {
      best = it->second.first;
    } else {
      double best_us = 1e30;
      for (int bn : {128, 256})
        for (int sp = 1; sp <= net->h_splits; ++sp) {
          TcPlan p;
          if (tc_plan_make(p, TC_SYRK, prec, net->Zt[0], net->Zt[1], n, net->K_total, net->Yt[0],
                           net->Yt[1], n, net->K_total, n, n, net->K_total, net->sm_count, bn,
                           sp) != NNC_OK)
            continue;
          if (p.splits != sp) continue;
          const double us = time_us(st, 3, [&] { tc_syrk(p, (float*)net->Hp, net->dev_err, st); });
          if (us < best_us) {
            best_us = us;
            best = bn * 1000 + sp;
          }
        }
      cache[key] = {best, best_us};
    }
    if (best != net->plan_syrk.bn * 1000 + net->plan_syrk.splits) {
      TcPlan p;
      if (!valid(best) ||
          tc_plan_make(p, TC_SYRK, prec, net->Zt[0], net->Zt[1], n, net->K_total, net->Yt[0],
                       net->Yt[1], n, net->K_total, n, n, net->K_total, net->sm_count, best / 1000,
                       best % 1000) != NNC_OK || p.splits > net->h_splits) {
        cache.erase(key);
        write_cache(cache_path, cache);
        set_last_error("autotune: the symmetric-product tiling " + std::to_string(best) +
                       " has no valid plan; the previous one is kept");
        return NNC_ERR_ARG;
      }
      net->plan_syrk = p;
    }
  }
  cudaStreamSynchronize(st);
  int e = 0;
  cudaMemcpy(&e, net->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) {
    int z = 0;
    cudaMemcpy(net->dev_err, &z, sizeof(int), cudaMemcpyHostToDevice);
    set_last_error("autotune: a bounded device-side wait ran out");
    return NNC_ERR_TIMEOUT;
  }
  write_cache(cache_path, cache);
  return cudaGetLastError() == cudaSuccess ? NNC_OK : NNC_ERR_CUDA;
}

extern "C" int nnc_tune_set(nnc_net* net, int tangent_bn, int syrk_splits) {
  if (!net) {
    set_last_error("net is NULL");
    return NNC_ERR_ARG;
  }
  const int prec = net->prec;
  if (!(prec == NNC_BF16 || prec == NNC_BF16X3 || prec == NNC_FP8)) return NNC_OK;  // CUDA-core forms
  {
    const int t = tangent_bn;
    const bool single = t == 112 || t == 128 || t == 208 || t == 256;
    const bool pair = t == -128 || t == -160 || t == -208 || t == -256;
    if (t == 1) {   // the persistent chain
      if (net->chain_nl <= 0) {
        set_last_error("this net has no persistent tangent chain (FP8 form, or too many layers)");
        return NNC_ERR_ARG;
      }
      if (syrk_splits < 0 || syrk_splits > net->h_splits) {
        set_last_error("symmetric-product splits out of range");
        return NNC_ERR_ARG;
      }
      net->use_chain = true;
      tangent_bn = 0;
    } else if (t && !single && !pair) {
      set_last_error("tangent tile must be 112, 128, 208, 256 (one SM), -128, -160, -208, -256 "
                     "(SM pairs) or 1 (the persistent chain)");
      return NNC_ERR_ARG;
    } else if (t) {
      net->use_chain = false;
    }
    if (pair && prec == NNC_FP8) {
      set_last_error("the SM-pair tangent kernel has no FP8 form");
      return NNC_ERR_ARG;
    }
  }
  if (syrk_splits < 0 || syrk_splits > net->h_splits) {
    set_last_error("symmetric-product splits out of range");
    return NNC_ERR_ARG;
  }
  cudaSetDevice(net->device);
  const int n = net->n_in;
  for (int l = 1; l < net->L && tangent_bn; ++l) {
    LayerDev& Ly = net->layers[l];
    if (!Ly.plan_tan.ready) continue;
    if (tangent_bn < 0 && Ly.mp % 256 != 0) continue;   // pairs need 256-row blocks
    const int cur = (l - 1) % 2;
    TcPlan p;
    const int r = prec == NNC_FP8
                      ? tc_plan_make(p, TC_TANGENT, prec, Ly.W8, nullptr, Ly.mp, Ly.kp, net->A8, nullptr,
                                     n, Ly.kp, Ly.mp, n, Ly.kp, net->sm_count, tangent_bn)
                      : tc_plan_make(p, TC_TANGENT, prec, Ly.Whi, Ly.Wlo, Ly.mp, Ly.kp, net->At[cur][0],
                                     net->At[cur][1], n, Ly.kp, Ly.mp, n, Ly.kp, net->sm_count,
                                     tangent_bn);
    if (r != NNC_OK) {
      set_last_error("tangent plan failed");
      return r;
    }
    Ly.plan_tan = p;
  }
  if (syrk_splits && net->K_total > 0 && net->plan_syrk.ready) {
    TcPlan p;
    const int r = tc_plan_make(p, TC_SYRK, prec, net->Zt[0], net->Zt[1], n, net->K_total, net->Yt[0],
                               net->Yt[1], n, net->K_total, n, n, net->K_total, net->sm_count, 0,
                               syrk_splits);
    if (r != NNC_OK || p.splits > net->h_splits) {
      set_last_error("symmetric-product plan failed");
      return r != NNC_OK ? r : NNC_ERR_ARG;
    }
    net->plan_syrk = p;
  }
  return NNC_OK;
}

extern "C" int nnc_tuning(const nnc_net* net, int layer, int* tangent_bn, int* syrk_splits) {
  if (!net || layer < 0 || layer >= net->L) {
    set_last_error("bad arguments");
    return NNC_ERR_ARG;
  }
  if (tangent_bn)
    *tangent_bn = !net->layers[layer].plan_tan.ready ? 0
                  : (net->use_chain && layer >= 1 && layer <= net->chain_nl) ? 1
                  : plan_code(net->layers[layer].plan_tan);
  if (syrk_splits) *syrk_splits = net->plan_syrk.ready ? net->plan_syrk.splits : net->h_splits;
  return NNC_OK;
}
