// Scheduling of the cubic kernels: size buckets, grid forms and the tuner.
//
// A batch's clusters, in decreasing-n order, fall into size buckets (dimension rounded up
// to 64).  Each cubic kernel (Cholesky, congruence, one-stage tridiagonalisation, band
// reduction, bulge chasing) is launched per bucket with that bucket's schedule: the grid
// form (one CTA per cluster, or a persistent grid of as many CTAs as fit the GPU taking
// clusters from an atomic work counter) and, in the mixed path, the tensor-core engine of
// the K <= 32 tile products (mma.sync or tcgen05).  All choices give the same bits: the
// arithmetic of a cluster does not depend on which CTA runs it, and both engines combine
// the same exact integer level sums.
//
// The tuner explores over solves: every eager solve of a batch (not one captured into a
// graph) times each (bucket, kernel) under its next untried candidate with CUDA events;
// once all candidates have been timed the fastest is kept.  Decisions are keyed by (GPU,
// precision, kernel, rounded dimension) in an optional text cache that later contexts
// read, so that they start with the tuned schedules.
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>

#include "dclno_internal.cuh"

static const char* kernel_name(int k) {
    static const char* names[TK_COUNT] = {"k_cholesky", "k_congruence", "k_tridiag", "k_band", "k_chase"};
    return names[k];
}

void build_buckets(dclno_ctx* c, Batch& b) {
    std::vector<Bucket> raw;
    for (int o = b.obeg; o < b.oend; ++o) {
        const int n = c->cl[c->order[o]].n;
        const int nr = (n + 63) / 64 * 64;
        if (raw.empty() || raw.back().nround != nr) {
            Bucket k;
            k.obeg = o;
            k.nround = nr;
            k.maxn = n;
            raw.push_back(k);
        }
        raw.back().oend = o + 1;
    }
    // a bucket below two CTAs per SM absorbs the next (smaller-n) one; a small last
    // bucket joins the one before it
    const int minc = c->bucket_min > 0 ? c->bucket_min : 2 * c->nsm;
    b.buckets.clear();
    for (const Bucket& k : raw) {
        if (!b.buckets.empty() && b.buckets.back().oend - b.buckets.back().obeg < minc) b.buckets.back().oend = k.oend;
        else b.buckets.push_back(k);
    }
    if (b.buckets.size() > 1 && b.buckets.back().oend - b.buckets.back().obeg < minc) {
        b.buckets[b.buckets.size() - 2].oend = b.buckets.back().oend;
        b.buckets.pop_back();
    }
}

static std::vector<Sched> candidates(const dclno_ctx* c, int kernel, bool mixed) {
    std::vector<Sched> v;
    const bool engine_kernel = mixed && (kernel == TK_CHOL || kernel == TK_CONG || kernel == TK_TRI);
    std::vector<int> engines;
    if (!mixed || kernel == TK_CHASE) engines = {0};
    else if (!engine_kernel) engines = {2};                // band reduction: long-K products on tcgen05
    else if (c->mixed_engine == 1 || c->mixed_engine == 2) engines = {c->mixed_engine};
    else engines = {1, 2};
    std::vector<int> forms;
    if (c->sched_force == 1) forms = {0};
    else if (c->sched_force == 2) forms = {1};
    else forms = {0, 1};
    for (int f : forms)
        for (int e : engines) v.push_back(Sched{e, f});
    return v;
}

// schedule before (or without) tuning: one CTA per cluster; mma.sync for the Cholesky and
// the one-stage tridiagonalisation, tcgen05 for the congruence (measured on the 1,728-atom
// step: 73 / 740 ms against 77 / 964 ms, and 254 against 254 ms)
static Sched default_sched(const dclno_ctx* c, int kernel, bool mixed) {
    const std::vector<Sched> v = candidates(c, kernel, mixed);
    int want_engine = !mixed ? 0 : (kernel == TK_CHOL || kernel == TK_TRI) ? 1 : 2;
    for (const Sched& s : v)
        if (s.engine == want_engine && s.persistent == (c->sched_force == 2 ? 1 : 0)) return s;
    return v.front();
}

// one tuner slot per (rounded dimension, kernel, precision), shared by the batches: a
// workload split into memory-admitted batches tunes once, timings compared per cluster
static std::string slot_key(const Batch& b, int k, int kernel, bool mixed) {
    return std::to_string(b.buckets[k].nround) + "/" + kernel_name(kernel) + "/" + (mixed ? "mixed" : "fp64");
}

static std::string cache_key(const dclno_ctx* c, int nround, int kernel, bool mixed) {
    return c->gpu_name + "|" + (mixed ? "mixed" : "fp64") + "|" + kernel_name(kernel) + "|" + std::to_string(nround);
}

static void save_cache(const dclno_ctx* c) {
    if (c->tune_cache_path.empty()) return;
    const std::string tmp = c->tune_cache_path + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return;
        f << "# libdclno schedule cache: gpu|precision|kernel|rounded-n engine persistent\n";
        for (const auto& kv : c->tune_cache) f << kv.first << " " << kv.second.engine << " " << kv.second.persistent << "\n";
    }
    std::rename(tmp.c_str(), c->tune_cache_path.c_str());
}

Sched sched_pick(dclno_ctx* c, const Batch& b, int k, int kernel, bool mixed, bool tune, int* cand) {
    *cand = -1;
    const std::vector<Sched> v = candidates(c, kernel, mixed);
    TuneSlot& slot = c->tune_slots[slot_key(b, k, kernel, mixed)];
    if ((int)slot.ms.size() != (int)v.size()) {
        slot = TuneSlot();
        slot.ms.assign(v.size(), -1.0f);
        const Sched d = default_sched(c, kernel, mixed);
        for (int i = 0; i < (int)v.size(); ++i)
            if (v[i].engine == d.engine && v[i].persistent == d.persistent) slot.default_index = i;
    }
    if (slot.chosen < 0 && c->sched_force == 0) {
        const auto it = c->tune_cache.find(cache_key(c, b.buckets[k].nround, kernel, mixed));
        if (it != c->tune_cache.end())
            for (int i = 0; i < (int)v.size(); ++i)
                if (v[i].engine == it->second.engine && v[i].persistent == it->second.persistent) {
                    slot.chosen = i;
                    slot.from_cache = true;
                }
    }
    if (slot.chosen >= 0) return v[slot.chosen];
    if (v.size() == 1) {
        slot.chosen = 0;
        return v[0];
    }
    if (!tune || !c->autotune || c->deferred || slot.next >= (int)v.size()) return default_sched(c, kernel, mixed);
    *cand = slot.next;
    return v[slot.next];
}

std::vector<SchedRun> sched_runs(dclno_ctx* c, const Batch& b, int kernel, bool mixed, bool tune,
                                 const std::vector<char>& use) {
    std::vector<SchedRun> runs;
    for (int k = 0; k < (int)b.buckets.size(); ++k) {
        if (!use[k]) continue;
        const Bucket& bk = b.buckets[k];
        SchedRun r;
        r.s = sched_pick(c, b, k, kernel, mixed, tune, &r.cand);
        r.k0 = k;
        r.k1 = k + 1;
        r.obeg = bk.obeg;
        r.oend = bk.oend;
        r.maxn = bk.maxn;
        SchedRun* last = runs.empty() ? nullptr : &runs.back();
        if (last && r.cand < 0 && last->cand < 0 && last->k1 == k && last->s.engine == r.s.engine &&
            last->s.persistent == r.s.persistent) {
            last->k1 = k + 1;
            last->oend = bk.oend;
            last->maxn = std::max(last->maxn, bk.maxn);
        } else {
            runs.push_back(r);
        }
    }
    return runs;
}

dclno_status sched_time_begin(dclno_ctx* c, cudaEvent_t* e0) {
    DCLNO_CUDA(c, cudaEventCreate(e0));
    DCLNO_CUDA(c, cudaEventRecord(*e0, c->stream));
    return DCLNO_OK;
}

dclno_status sched_time_end(dclno_ctx* c, const Batch& b, int k, int kernel, bool mixed, int cand, cudaEvent_t e0) {
    cudaEvent_t e1;
    DCLNO_CUDA(c, cudaEventCreate(&e1));
    DCLNO_CUDA(c, cudaEventRecord(e1, c->stream));
    c->tune_pending.push_back(TunePending{slot_key(b, k, kernel, mixed), cand, e0, e1,
                                          b.buckets[k].oend - b.buckets[k].obeg});
    return DCLNO_OK;
}

void sched_collect(dclno_ctx* c) {
    for (TunePending& p : c->tune_pending) {
        float ms = -1.0f;
        if (cudaEventSynchronize(p.e1) != cudaSuccess || cudaEventElapsedTime(&ms, p.e0, p.e1) != cudaSuccess) ms = -1.0f;
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
        auto it = c->tune_slots.find(p.slot);
        if (it == c->tune_slots.end() || ms < 0.0f) continue;
        TuneSlot& s = it->second;
        if (p.cand < 0 || p.cand >= (int)s.ms.size() || s.chosen >= 0) continue;
        s.ms[p.cand] = ms / (float)std::max(p.clusters, 1);
        s.next = std::max(s.next, p.cand + 1);
        if (s.next >= (int)s.ms.size()) {
            int best = 0;
            for (int i = 1; i < (int)s.ms.size(); ++i)
                if (s.ms[i] >= 0.0f && (s.ms[best] < 0.0f || s.ms[i] < s.ms[best])) best = i;
            // the default stays unless another schedule is 2% faster: a difference within
            // run-to-run noise would split launches (and tails) for nothing
            const int d = s.default_index;
            if (d >= 0 && d < (int)s.ms.size() && s.ms[d] >= 0.0f && s.ms[d] <= 1.02f * s.ms[best]) best = d;
            s.chosen = best;
        }
    }
    c->tune_pending.clear();
    // newly decided slots go to the cache
    bool dirty = false;
    for (const Batch& b : c->batches)
        for (int k = 0; k < (int)b.buckets.size(); ++k)
            for (int kernel = 0; kernel < TK_COUNT; ++kernel)
                for (int mixed = 0; mixed < 2; ++mixed) {
                    auto it = c->tune_slots.find(slot_key(b, k, kernel, mixed != 0));
                    if (it == c->tune_slots.end() || it->second.chosen < 0 || it->second.from_cache ||
                        it->second.ms.size() < 2)
                        continue;
                    const std::vector<Sched> v = candidates(c, kernel, mixed != 0);
                    if (it->second.chosen >= (int)v.size()) continue;
                    const std::string ck = cache_key(c, b.buckets[k].nround, kernel, mixed != 0);
                    const Sched s = v[it->second.chosen];
                    auto old = c->tune_cache.find(ck);
                    if (old == c->tune_cache.end() || old->second.engine != s.engine ||
                        old->second.persistent != s.persistent) {
                        c->tune_cache[ck] = s;
                        dirty = true;
                    }
                }
    if (dirty) save_cache(c);
}

void sched_reset(dclno_ctx* c) {
    for (TunePending& p : c->tune_pending) {
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    c->tune_pending.clear();
    c->tune_slots.clear();
}

int sched_grid(dclno_ctx* c, const void* fn, int threads, size_t smem, int nitems, bool persistent) {
    if (!persistent) return nitems;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return std::max(1, std::min(nitems, per_sm * c->nsm));
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" dclno_status dclno_set_schedule(dclno_ctx* c, int mode) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (mode < 0 || mode > 2) return set_err(c, DCLNO_ERR_ARG, "dclno_set_schedule: mode must be 0, 1 or 2");
    c->sched_force = mode;
    sched_reset(c);
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_bucket_min(dclno_ctx* c, int count) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    if (count < 0) return set_err(c, DCLNO_ERR_ARG, "dclno_set_bucket_min: count must be >= 0");
    c->bucket_min = count;
    for (Batch& b : c->batches) build_buckets(c, b);
    sched_reset(c);
    return DCLNO_OK;
}

extern "C" dclno_status dclno_set_tuning_cache(dclno_ctx* c, const char* path) {
    if (!c) return DCLNO_ERR_ARG;
    c->err.clear();
    c->tune_cache.clear();
    c->tune_cache_path = path ? path : "";
    if (!path) return DCLNO_OK;
    std::ifstream f(path);
    if (!f) return DCLNO_OK;  // a cache that does not exist yet
    std::string line;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        std::string key;
        Sched s;
        if (is >> key >> s.engine >> s.persistent && s.engine >= 0 && s.engine <= 2 && (s.persistent == 0 || s.persistent == 1))
            c->tune_cache[key] = s;
    }
    sched_reset(c);
    return DCLNO_OK;
}

extern "C" dclno_status dclno_tuning_report(dclno_ctx* c, char* buf, size_t len, size_t* needed) {
    if (!c) return DCLNO_ERR_ARG;
    std::ostringstream o;
    o << "{\"gpu\": \"" << c->gpu_name << "\", \"batches\": [";
    for (size_t bi = 0; bi < c->batches.size(); ++bi) {
        const Batch& b = c->batches[bi];
        o << (bi ? ", " : "") << "{\"buckets\": [";
        for (size_t k = 0; k < b.buckets.size(); ++k) {
            const Bucket& bk = b.buckets[k];
            o << (k ? ", " : "") << "{\"n_rounded\": " << bk.nround << ", \"clusters\": " << (bk.oend - bk.obeg)
              << ", \"schedules\": {";
            bool first = true;
            for (int mixed = 0; mixed < 2; ++mixed)
                for (int kernel = 0; kernel < TK_COUNT; ++kernel) {
                    auto it = c->tune_slots.find(slot_key(b, (int)k, kernel, mixed != 0));
                    if (it == c->tune_slots.end()) continue;
                    const std::vector<Sched> v = candidates(c, kernel, mixed != 0);
                    const TuneSlot& s = it->second;
                    const Sched sc = s.chosen >= 0 && s.chosen < (int)v.size() ? v[s.chosen]
                                                                                 : default_sched(c, kernel, mixed != 0);
                    o << (first ? "" : ", ") << "\"" << kernel_name(kernel) << (mixed ? "/mixed" : "/fp64")
                      << "\": {\"engine\": " << sc.engine << ", \"persistent\": " << sc.persistent
                      << ", \"decided\": " << (s.chosen >= 0 ? "true" : "false")
                      << ", \"from_cache\": " << (s.from_cache ? "true" : "false") << ", \"ms\": [";
                    for (size_t i = 0; i < s.ms.size(); ++i) o << (i ? ", " : "") << s.ms[i];
                    o << "]}";
                    first = false;
                }
            o << "}}";
        }
        o << "]}";
    }
    o << "]}";
    const std::string r = o.str();
    if (needed) *needed = r.size() + 1;
    if (buf && len) {
        const size_t m = std::min(len - 1, r.size());
        std::copy(r.begin(), r.begin() + m, buf);
        buf[m] = '\0';
    }
    return DCLNO_OK;
}
