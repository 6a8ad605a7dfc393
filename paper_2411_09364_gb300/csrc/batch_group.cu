// Grouped execution of a batch of FP32 + refinement solves: one launch per
// stage (and kernel variant) for all solves of the batch; see batch_group.h.
#include <algorithm>
#include <cstring>
#include <map>
#include <set>

#include "batch_group.h"
#include "cales.h"

using namespace cales;

namespace {

enum StageKind { SK_XFWD64, SK_XFWD32, SK_YFWD, SK_YINV, SK_Z, SK_XINV, SK_RESID, SK_ZERO_ALL, SK_ZERO_GAUGE };

struct Launch {
    int kind;
    int variant;       // y: tile width; z: segment bound; x inverse: output mode; residual: variant bits
    size_t arg_off;    // byte offsets of the argument blocks and the work list in the device buffer
    size_t work_off;
    int nblocks;
    size_t smem;
    int threads;
};

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename A> size_t push_bytes(std::vector<unsigned char>& hb, const A* p, size_t count) {
    const size_t off = align16(hb.size());
    hb.resize(off + count * sizeof(A));
    std::memcpy(hb.data() + off, p, count * sizeof(A));
    return off;
}

long cdiv(long a, long b) { return (a + b - 1) / b; }

}  // namespace

struct GroupedBatch {
    std::vector<const void*> f;
    std::vector<void*> u;
    unsigned char* dev = nullptr;    // argument blocks and work lists
    double* acc = nullptr;           // [2n]: consistency constants, then gauge sums
    int n = 0;
    bool any_singular = false;
    std::vector<Launch> launches;
};

namespace {

// One launch of `args` (one argument block per item; blocks[i] CTAs each),
// largest items first in the work list.
template <typename A>
void add_launch(GroupedBatch* G, std::vector<unsigned char>& hb, int kind, int variant, const std::vector<A>& args,
                const std::vector<long>& blocks, size_t smem, int threads) {
    if (args.empty()) return;
    std::vector<int> order(args.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return blocks[a] > blocks[b]; });
    std::vector<int2> work;
    for (int i : order)
        for (long b = 0; b < blocks[i]; ++b) work.push_back(make_int2(i, (int)b));
    Launch L;
    L.kind = kind;
    L.variant = variant;
    L.arg_off = push_bytes(hb, args.data(), args.size());
    L.work_off = push_bytes(hb, work.data(), work.size());
    L.nblocks = (int)work.size();
    L.smem = smem;
    L.threads = threads;
    G->launches.push_back(L);
}

struct Item {
    cales_plan_t P;
    bool helm;
    double alpha;
    const void* f;
    void* u;
    PassOpt o;
};

// The five stages of one pass over every item: in (the right-hand side on
// the first pass, else the residual in the plan's work field) -> mode space
// -> out (the pair field / FP64 result) with output mode `mode`.
void add_pass(GroupedBatch* G, std::vector<unsigned char>& hb, std::vector<Item>& it, bool first, int mode) {
    const size_t n = it.size();
    {   // x forward
        std::vector<RowArgs<float>> a(n);
        std::vector<long> nb(n);
        size_t sm = 0;
        for (size_t i = 0; i < n; ++i) {
            cales_plan_t P = it[i].P;
            a[i] = first ? fwd_row_args<float, double>(P, it[i].f, P->work) : fwd_row_args<float, float>(P, P->work, P->work);
            nb[i] = cdiv(a[i].nrows, a[i].rpc);
            sm = std::max(sm, rows_smem_bytes<float>(a[i]));
        }
        add_launch(G, hb, first ? SK_XFWD64 : SK_XFWD32, 0, a, nb, sm, 256);
    }
    // y forward / inverse, one launch per tile width
    std::map<int, std::vector<int>> by_tx;
    std::vector<ColArgs<float>> ca(n);
    for (size_t i = 0; i < n; ++i) {
        ca[i] = col_args<float>(it[i].P, it[i].P->work);
        if (it[i].P->ny > 1) by_tx[ca[i].tx].push_back((int)i);
    }
    auto add_cols = [&](bool inverse) {
        for (const auto& kv : by_tx) {
            std::vector<ColArgs<float>> a;
            std::vector<long> nb;
            size_t sm = 0;
            for (int i : kv.second) {
                a.push_back(ca[i]);
                nb.push_back(ca[i].nplanes * cdiv(ca[i].nx, ca[i].tx));
                sm = std::max(sm, cols_smem_bytes<float>(ca[i]));
            }
            add_launch(G, hb, inverse ? SK_YINV : SK_YFWD, kv.first, a, nb, sm, 256);
        }
    };
    add_cols(false);
    {   // z, one launch per segment bound; CTAs of shallower lines leave the
        // warps beyond their segment count idle (measured on the 16-domain
        // substep: 2.7 ms per substep for the z stages, against 3.3 ms with a
        // launch per segment count, whose extra launch tails cost more)
        std::map<int, std::vector<ZArgs<float>>> by_m;
        std::map<int, std::vector<long>> nb_m;
        std::map<int, int> pmax;
        for (size_t i = 0; i < n; ++i) {
            ZArgs<float> za = z_args<float>(it[i].P, it[i].P->work, it[i].o);
            z_args_done<float>(it[i].P, za, it[i].o);
            by_m[za.maxm].push_back(za);
            nb_m[za.maxm].push_back(cdiv((long)za.nx * za.ny, 32));
            pmax[za.maxm] = std::max(pmax[za.maxm], za.P);
        }
        for (auto& kv : by_m) {
            const int pb = pmax[kv.first];
            size_t sm = 0;
            for (const auto& za : kv.second) sm = std::max(sm, zsolve_w_smem_pb<float>(za.nz, za.P, pb));
            add_launch(G, hb, SK_Z, kv.first, kv.second, nb_m[kv.first], sm, 32 * pb);
        }
    }
    add_cols(true);
    {   // x inverse
        std::vector<RowArgs<float>> a(n);
        std::vector<long> nb(n);
        size_t sm = 0;
        for (size_t i = 0; i < n; ++i) {
            cales_plan_t P = it[i].P;
            switch (mode) {
                case OUT_F64: a[i] = inv_row_args<float, OUT_F64>(P, P->work, it[i].u, it[i].o); break;
                case OUT_FF_INIT: a[i] = inv_row_args<float, OUT_FF_INIT>(P, P->work, it[i].u, it[i].o); break;
                case OUT_FF_ACC: a[i] = inv_row_args<float, OUT_FF_ACC>(P, P->work, it[i].u, it[i].o); break;
                default: a[i] = inv_row_args<float, OUT_FF_FINAL>(P, P->work, it[i].u, it[i].o); break;
            }
            nb[i] = cdiv(a[i].nrows, a[i].rpc);
            sm = std::max(sm, rows_smem_bytes<float>(a[i]));
        }
        add_launch(G, hb, SK_XINV, mode, a, nb, sm, 256);
    }
}

bool aligned(const void* p, unsigned a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

GroupedBatch* grouped_build(const std::vector<cales_plan_t>& plans, const std::vector<int>& kinds,
                            const std::vector<double>& alphas, const void* const* f, void* const* u, int* rc) {
    *rc = CALES_OK;
    const size_t n = plans.size();
    if (n == 0) return nullptr;
    std::set<cales_plan_t> seen;
    const int ns = plans[0]->sweeps;
    for (size_t i = 0; i < n; ++i) {
        cales_plan_t P = plans[i];
        if (!P || P->precision != CALES_FP32_REFINE || P->sweeps != ns || !P->work || P->bc[4] == CALES_BC_P) return nullptr;
        if (!seen.insert(P).second) return nullptr;            // solves of one plan share its workspace
        if (!f[i] || !u[i] || f[i] == u[i]) return nullptr;
        // the grouped residual is the vector kernel: even rows, 16-byte aligned fields
        if (ns > 0 && (P->nx % 2 || !aligned(f[i], 16) || !aligned(u[i], 16))) return nullptr;
        ZArgs<float> za = z_args<float>(P, P->work, solve_opts(P, kinds[i] == 1, alphas[i], false));
        if (!za.warp_mode || za.P > 16) return nullptr;
    }
    GroupedBatch* G = new GroupedBatch();
    G->n = (int)n;
    G->f.assign(f, f + n);
    G->u.assign(u, u + n);
    if (cudaMalloc(&G->acc, 2 * n * sizeof(double)) != cudaSuccess) {
        delete G;
        *rc = CALES_ENOMEM;
        return nullptr;
    }
    std::vector<Item> it(n);
    for (size_t i = 0; i < n; ++i) {
        cales_plan_t P = plans[i];
        it[i].P = P;
        it[i].helm = kinds[i] == 1;
        it[i].alpha = alphas[i];
        it[i].f = f[i];
        it[i].u = u[i];
        it[i].o = solve_opts(P, it[i].helm, it[i].alpha, false);
        if (it[i].o.singular) {
            it[i].o.cacc = G->acc + i;
            G->any_singular = true;
        }
    }
    std::vector<unsigned char> hb;
    {   // accumulators start at zero
        Launch L{SK_ZERO_ALL, 0, 0, 0, 0, 0, 0};
        G->launches.push_back(L);
    }
    add_pass(G, hb, it, true, ns == 0 ? OUT_F64 : OUT_FF_INIT);
    for (int s = 0; s < ns; ++s) {
        if (G->any_singular) {
            Launch L{SK_ZERO_GAUGE, 0, 0, 0, 0, 0, 0};
            G->launches.push_back(L);
        }
        std::map<int, std::vector<ResidFFArgs>> by_v;
        std::map<int, std::vector<long>> nb_v;
        for (size_t i = 0; i < n; ++i) {
            cales_plan_t P = it[i].P;
            const ResidFFArgs ra = resid_args(P, it[i].helm, it[i].alpha, f[i], u[i], P->work, G->acc + i,
                                              G->acc + n + i, s, ns);
            const int v = (ra.cshift ? 1 : 0) | (it[i].helm ? 2 : 0) | (ra.gacc ? 4 : 0) | (ra.lo_zero ? 0 : 8);
            by_v[v].push_back(ra);
            nb_v[v].push_back(cdiv(P->ny, ra.rows_per_cta) * P->nz);
        }
        for (auto& kv : by_v) add_launch(G, hb, SK_RESID, kv.first, kv.second, nb_v[kv.first], 0, 256);
        for (size_t i = 0; i < n; ++i) {
            const bool last = s == ns - 1;
            it[i].o.shift_acc = (it[i].o.singular && last) ? G->acc + n + i : nullptr;
            it[i].o.shift_scale = 1.0 / ((double)it[i].P->nx * (double)it[i].P->ny * it[i].P->dzf_sum);
        }
        add_pass(G, hb, it, false, s == ns - 1 ? OUT_FF_FINAL : OUT_FF_ACC);
    }
    if (cudaMalloc(&G->dev, hb.size() + 16) != cudaSuccess ||
        cudaMemcpy(G->dev, hb.data(), hb.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        grouped_free(G);
        *rc = CALES_ECUDA;
        return nullptr;
    }
    return G;
}

bool grouped_same_buffers(const GroupedBatch* g, const void* const* f, void* const* u) {
    if (!g) return false;
    for (int i = 0; i < g->n; ++i)
        if (g->f[i] != f[i] || g->u[i] != u[i]) return false;
    return true;
}

int grouped_enqueue(GroupedBatch* G, cudaStream_t st) {
    for (const Launch& L : G->launches) {
        cudaError_t e = cudaSuccess;
        const unsigned char* args = G->dev + L.arg_off;
        const int2* work = reinterpret_cast<const int2*>(G->dev + L.work_off);
        switch (L.kind) {
            case SK_ZERO_ALL: e = cudaMemsetAsync(G->acc, 0, 2 * (size_t)G->n * sizeof(double), st); break;
            case SK_ZERO_GAUGE: e = cudaMemsetAsync(G->acc + G->n, 0, (size_t)G->n * sizeof(double), st); break;
            case SK_XFWD64:
                e = launch_rows_forward_grp<float, double>(reinterpret_cast<const RowArgs<float>*>(args), work,
                                                           L.nblocks, L.smem, st);
                break;
            case SK_XFWD32:
                e = launch_rows_forward_grp<float, float>(reinterpret_cast<const RowArgs<float>*>(args), work,
                                                          L.nblocks, L.smem, st);
                break;
            case SK_YFWD:
            case SK_YINV:
                e = launch_cols_grp<float>(reinterpret_cast<const ColArgs<float>*>(args), work, L.nblocks, L.variant,
                                           L.kind == SK_YINV, L.smem, st);
                break;
            case SK_Z:
                e = launch_zsolve_grp<float>(reinterpret_cast<const ZArgs<float>*>(args), work, L.nblocks, L.variant,
                                             false, L.threads, L.smem, st);
                break;
            case SK_XINV: {
                const RowArgs<float>* a = reinterpret_cast<const RowArgs<float>*>(args);
                switch (L.variant) {
                    case OUT_F64: e = launch_rows_inverse_grp<float, OUT_F64>(a, work, L.nblocks, L.smem, st); break;
                    case OUT_FF_INIT: e = launch_rows_inverse_grp<float, OUT_FF_INIT>(a, work, L.nblocks, L.smem, st); break;
                    case OUT_FF_ACC: e = launch_rows_inverse_grp<float, OUT_FF_ACC>(a, work, L.nblocks, L.smem, st); break;
                    default: e = launch_rows_inverse_grp<float, OUT_FF_FINAL>(a, work, L.nblocks, L.smem, st); break;
                }
                break;
            }
            case SK_RESID:
                e = launch_residual_ff_grp(reinterpret_cast<const ResidFFArgs*>(args), work, L.nblocks, L.variant, st);
                break;
            default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return CALES_ECUDA;
    }
    return CALES_OK;
}

int grouped_launches(const GroupedBatch* g) { return g ? (int)g->launches.size() : 0; }

void grouped_free(GroupedBatch* g) {
    if (!g) return;
    if (g->dev) cudaFree(g->dev);
    if (g->acc) cudaFree(g->acc);
    delete g;
}
