// Batched solves in one CUDA graph, and the schedule autotuner.
//
// A Runge-Kutta substep of the paper's fractional-step method (Algorithm 1,
// Sec. 2.2) needs, per domain, the three Crank-Nicolson Helmholtz solves of
// Eq. (18) and the Poisson solve of Eq. (12); a set of independent domains
// multiplies that.  The batch executor forks the solves over several streams
// (solves that share a plan stay on one stream, since they share its
// workspace), balancing the streams by grid size, joins them back on the
// caller's stream, and can capture the whole fork/join into one CUDA graph
// that is replayed with a single launch.
//
// The autotuner times candidate launch schedules of one plan on the device
// (x shared-memory budget, y tile width, z warps and segment length), keeps
// the fastest per stage, and caches the result in a small JSON file keyed by
// grid, boundary kinds, precision and device name.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "batch_group.h"
#include "cales.h"
#include "plan.h"

struct cales_batch_s {
    GroupedBatch* grp = nullptr;       // grouped stage launches for the last buffers (nullptr: fork/join)
    int grouped = 1;                   // try grouped launches (cales_batch_set_grouped)
    int used_grouped = 0;              // the last solve / capture used them
    std::vector<cales_plan_t> plans;
    std::vector<int> kinds;
    std::vector<double> alphas;
    std::vector<int> stream_of;        // solve -> stream index
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void destroy_graph(cales_batch_s* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
}

int enqueue(cales_batch_s* B, const void* const* f, void* const* u, cudaStream_t st) {
    if (cudaEventRecord(B->fork, st) != cudaSuccess) return CALES_ECUDA;
    for (cudaStream_t s : B->streams)
        if (cudaStreamWaitEvent(s, B->fork, 0) != cudaSuccess) return CALES_ECUDA;
    for (size_t i = 0; i < B->plans.size(); ++i) {
        const int rc = cales_internal_solve(B->plans[i], B->kinds[i] == 1, B->alphas[i], false, f[i], u[i],
                                            B->streams[B->stream_of[i]]);
        if (rc) return rc;
    }
    for (size_t k = 0; k < B->streams.size(); ++k) {
        if (cudaEventRecord(B->join[k], B->streams[k]) != cudaSuccess) return CALES_ECUDA;
        if (cudaStreamWaitEvent(st, B->join[k], 0) != cudaSuccess) return CALES_ECUDA;
    }
    return CALES_OK;
}

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

std::string tune_key(cales_plan_t P) {
    char buf[256];
    snprintf(buf, sizeof buf, "%d,%d,%d,%d,%d,%d,%d,%d,%s", P->nx, P->ny, P->nz, P->X.kind, P->Y.kind, P->bc[4],
             P->bc[5], P->precision, device_name().c_str());
    return buf;
}

std::map<std::string, std::vector<int>> read_cache(const char* path) {
    std::map<std::string, std::vector<int>> m;
    FILE* fp = path ? fopen(path, "r") : nullptr;
    if (!fp) return m;
    char line[1024];
    while (fgets(line, sizeof line, fp)) {
        char* q1 = strchr(line, '"');
        if (!q1) continue;
        char* q2 = strchr(q1 + 1, '"');
        if (!q2) continue;
        std::string key(q1 + 1, q2);
        int v[6] = {0, 0, 0, 0, 0, 0};
        char* br = strchr(q2, '[');
        const int got = br ? sscanf(br, "[%d,%d,%d,%d,%d,%d]", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) : 0;
        if (got == 4 || got == 6) m[key] = {v[0], v[1], v[2], v[3], v[4], v[5]};
    }
    fclose(fp);
    return m;
}

bool write_cache(const char* path, const std::map<std::string, std::vector<int>>& m) {
    FILE* fp = fopen(path, "w");
    if (!fp) return false;
    fprintf(fp, "{\n");
    size_t i = 0;
    for (const auto& kv : m) {
        fprintf(fp, "  \"%s\": [%d,%d,%d,%d,%d,%d]%s\n", kv.first.c_str(), kv.second[0], kv.second[1],
                kv.second[2], kv.second[3], kv.second[4], kv.second[5], ++i < m.size() ? "," : "");
    }
    fprintf(fp, "}\n");
    fclose(fp);
    return true;
}

// Median-free timing: sum of the per-stage event times of `reps` solves.
int stage_times(cales_plan_t P, const void* f, void* p, cudaStream_t st, int reps, double t[3]) {
    const bool was = P->prof_on;
    P->prof_on = true;
    P->prof_n = 0;
    int rc = CALES_OK;
    for (int r = 0; r < reps && rc == CALES_OK; ++r) rc = cales_internal_solve(P, false, 0.0, false, f, p, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = CALES_ECUDA;
    t[0] = t[1] = t[2] = 0.0;
    for (int i = 0; i < P->prof_n; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, P->prof[i].a, P->prof[i].b);
        const char* n = P->prof[i].name;
        const int stage = n[0] == 'x' ? 0 : (n[0] == 'y' ? 1 : (n[0] == 'z' ? 2 : -1));
        if (stage >= 0) t[stage] += ms;
    }
    P->prof_on = was;
    P->prof_n = 0;
    return rc;
}

}  // namespace

extern "C" {

int cales_set_schedule(cales_plan_t P, const int sched[CALES_SCHED_LEN]) {
    if (!P || !sched) return CALES_EINVAL;
    for (int i = 0; i < CALES_SCHED_LEN; ++i)
        if (sched[i] < 0) return CALES_EINVAL;
    if (sched[4] > 2 || sched[5] > 1) return CALES_EINVAL;
    const int rc = plan_set_radix_order(P, sched[4]);
    if (rc) return rc;
    for (int i = 0; i < CALES_SCHED_LEN; ++i) P->sched[i] = sched[i];
    return CALES_OK;
}

int cales_get_schedule(cales_plan_t P, int sched[CALES_SCHED_LEN]) {
    if (!P || !sched) return CALES_EINVAL;
    for (int i = 0; i < CALES_SCHED_LEN; ++i) sched[i] = P->sched[i];
    return CALES_OK;
}

int cales_autotune(cales_plan_t P, const char* cache_path, void* stream) {
    if (!P) return CALES_EINVAL;
    const std::string key = tune_key(P);
    auto cache = read_cache(cache_path);
    auto it = cache.find(key);
    if (it != cache.end()) return cales_set_schedule(P, it->second.data());

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)P->nx * P->ny * P->nz;
    const size_t esz = P->precision == CALES_FP32 ? 4 : 8;
    void *f = nullptr, *p = nullptr;
    if (cudaMalloc(&f, n * esz) != cudaSuccess) return CALES_ENOMEM;
    if (cudaMalloc(&p, n * esz) != cudaSuccess) { cudaFree(f); return CALES_ENOMEM; }
    cudaMemsetAsync(f, 0, n * esz, st);
    int best[CALES_SCHED_LEN] = {0, 0, 0, 0, 0, 0};
    int rc = cales_set_schedule(P, best);
    double t[3];
    rc = rc ? rc : stage_times(P, f, p, st, 1, t);      // warm-up
    // time a candidate: knobs k1 (and k2) changed from the best so far; false
    // when the schedule is refused or a launch fails
    auto trial = [&](int k1, int v1, int k2, int v2, double out[3]) {
        int s[CALES_SCHED_LEN];
        for (int i = 0; i < CALES_SCHED_LEN; ++i) s[i] = best[i];
        s[k1] = v1;
        if (k2 >= 0) s[k2] = v2;
        out[0] = out[1] = out[2] = 1e30;
        if (rc || cales_set_schedule(P, s) != CALES_OK) return false;
        rc = stage_times(P, f, p, st, 1, out);            // first run with a new schedule fills caches
        if (!rc) rc = stage_times(P, f, p, st, 3, out);
        return rc == CALES_OK;
    };
    // FFT radix order (x and y stages together)
    {
        double bt = 1e30;
        for (int c = 0; c <= 2; ++c)
            if (trial(4, c, -1, 0, t) && t[0] + t[1] < bt) { bt = t[0] + t[1]; best[4] = c; }
    }
    // x: shared-memory budget per CTA
    {
        double bt = 1e30;
        const int cand[3] = {32, 64, 96};
        for (int c : cand)
            if (trial(0, c, -1, 0, t) && t[0] < bt) { bt = t[0]; best[0] = c; }
    }
    // y: tile width
    if (P->ny > 1) {
        double bt = 1e30;
        const int cand[6] = {8, 16, 32, 64, 128, 0};
        for (int c : cand)
            if (trial(1, c, -1, 0, t) && t[1] < bt) { bt = t[1]; best[1] = c; }
    }
    // z: warps x segment bound, then the kernel variant (kept only when it
    // wins by more than 3 %)
    {
        double bt = 1e30;
        int bw = 0, bm = 0;
        const int mms[3] = {16, 32, 64};
        for (int mm : mms) {
            const int w = (P->nz + mm - 1) / mm;
            if (w < 1 || w > 16) continue;
            if (trial(2, w, 3, mm, t) && t[2] < bt) { bt = t[2]; bw = w; bm = mm; }
        }
        best[2] = bw;
        best[3] = bm;
        double tz[3];
        if (trial(5, 1, -1, 0, tz) && tz[2] < 0.97 * bt) best[5] = 1;
    }
    cudaFree(f);
    cudaFree(p);
    if (rc) {
        int zero[CALES_SCHED_LEN] = {0, 0, 0, 0, 0, 0};
        cales_set_schedule(P, zero);
        return rc;
    }
    rc = cales_set_schedule(P, best);
    if (rc) return rc;
    if (cache_path) {
        cache[key] = std::vector<int>(best, best + CALES_SCHED_LEN);
        write_cache(cache_path, cache);
    }
    return CALES_OK;
}

int cales_batch_create(cales_batch_t* out, int n, const cales_plan_t* plans, const int* kinds, const double* alphas) {
    if (!out || n < 1 || !plans || !kinds) return CALES_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || (kinds[i] != 0 && kinds[i] != 1)) return CALES_EINVAL;
        if (kinds[i] == 1 && !(alphas && alphas[i] > 0.0)) return CALES_EINVAL;
    }
    cales_batch_s* B = new cales_batch_s();
    B->plans.assign(plans, plans + n);
    B->kinds.assign(kinds, kinds + n);
    B->alphas.assign(n, 0.0);
    if (alphas)
        for (int i = 0; i < n; ++i) B->alphas[i] = kinds[i] == 1 ? alphas[i] : 0.0;
    // group solves by plan (shared workspace), then place groups on the
    // least-loaded stream, largest first
    std::map<cales_plan_t, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) groups[plans[i]].push_back(i);
    std::vector<std::pair<double, cales_plan_t>> order;
    for (const auto& g : groups)
        order.push_back({(double)g.first->nx * g.first->ny * g.first->nz * g.second.size(), g.first});
    std::sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    const int ns = std::min<int>((int)order.size(), 8);
    std::vector<double> load(ns, 0.0);
    B->stream_of.assign(n, 0);
    for (const auto& o : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += o.first;
        for (int i : groups[o.second]) B->stream_of[i] = k;
    }
    int rc = CALES_OK;
    B->streams.resize(ns);
    B->join.resize(ns);
    for (int k = 0; k < ns && !rc; ++k) {
        if (cudaStreamCreateWithFlags(&B->streams[k], cudaStreamNonBlocking) != cudaSuccess) rc = CALES_ECUDA;
        if (cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming) != cudaSuccess) rc = CALES_ECUDA;
    }
    if (!rc && cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) rc = CALES_ECUDA;
    if (rc) {
        cales_batch_destroy(B);
        return rc;
    }
    *out = B;
    return CALES_OK;
}

// The grouped launches for buffers f -> u (built on first use, rebuilt when
// the buffers change); nullptr when the batch takes the fork/join path.
static int prepare_grouped(cales_batch_t B, const void* const* f, void* const* u) {
    B->used_grouped = 0;
    if (!B->grouped) return CALES_OK;
    if (!grouped_same_buffers(B->grp, f, u)) {
        grouped_free(B->grp);
        int rc = CALES_OK;
        B->grp = grouped_build(B->plans, B->kinds, B->alphas, f, u, &rc);
        if (rc) return rc;
    }
    B->used_grouped = B->grp ? 1 : 0;
    return CALES_OK;
}

int cales_batch_solve(cales_batch_t B, const void* const* f, void* const* u, void* stream) {
    if (!B || !f || !u) return CALES_EINVAL;
    const int rc = prepare_grouped(B, f, u);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return B->used_grouped ? grouped_enqueue(B->grp, st) : enqueue(B, f, u, st);
}

int cales_batch_set_grouped(cales_batch_t B, int on) {
    if (!B) return CALES_EINVAL;
    B->grouped = on ? 1 : 0;
    if (!on) {
        grouped_free(B->grp);
        B->grp = nullptr;
    }
    return CALES_OK;
}

int cales_batch_grouped(cales_batch_t B, int* used) {
    if (!B || !used) return CALES_EINVAL;
    *used = B->used_grouped;
    return CALES_OK;
}

int cales_batch_capture(cales_batch_t B, const void* const* f, void* const* u, void* stream) {
    if (!B || !f || !u || !stream) return CALES_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    destroy_graph(B);
    const int prc = prepare_grouped(B, f, u);       // uploads argument blocks: before the capture
    if (prc) return prc;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CALES_ECUDA;
    const int rc = B->used_grouped ? grouped_enqueue(B->grp, st) : enqueue(B, f, u, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return CALES_ECUDA;
    B->graph = g;
    if (cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) {
        destroy_graph(B);
        return CALES_ECUDA;
    }
    return CALES_OK;
}

int cales_batch_launch(cales_batch_t B, void* stream) {
    if (!B || !B->exec) return CALES_EINVAL;
    return cudaGraphLaunch(B->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? CALES_OK : CALES_ECUDA;
}

int cales_batch_graph_nodes(cales_batch_t B, unsigned long* nodes) {
    if (!B || !B->graph || !nodes) return CALES_EINVAL;
    size_t n = 0;
    if (cudaGraphGetNodes(B->graph, nullptr, &n) != cudaSuccess) return CALES_ECUDA;
    *nodes = (unsigned long)n;
    return CALES_OK;
}

void cales_batch_destroy(cales_batch_t B) {
    if (!B) return;
    destroy_graph(B);
    grouped_free(B->grp);
    for (cudaStream_t s : B->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->join)
        if (e) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    delete B;
}

}  // extern "C"
