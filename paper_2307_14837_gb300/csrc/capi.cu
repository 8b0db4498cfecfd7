// extern "C" entry points of libdnnmg (declared in include/dnnmg.h).
#include <chrono>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <new>
#include <thread>

#include "internal.h"

using namespace dnnmg;

#include <nvtx3/nvToolsExt.h>

namespace {

// An NVTX range over one entry point (a no-op unless a profiler is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

const char* kStatusText[] = {"ok", "invalid argument", "out of memory", "CUDA error", "no convergence",
                             "NaN or Inf", "timeout", "call out of order", "unsupported"};

dnnmg_status fail(dnnmg_ctx* ctx, dnnmg_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

dnnmg_status cuda_fail(dnnmg_ctx* ctx, cudaError_t e, const char* where) {
    if (ctx) ctx->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DNNMG_ENOMEM : DNNMG_ECUDA;
}

#define CK(ctx, call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <typename T>
dnnmg_status upload(dnnmg_ctx* ctx, const T* host, size_t n, T** dev) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T) > 0 ? n * sizeof(T) : 1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    ctx->allocations.push_back(p);
    if (n) {
        e = cudaMemcpy(p, host, n * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
    }
    *dev = static_cast<T*>(p);
    return DNNMG_OK;
}

dnnmg_status alloc(dnnmg_ctx* ctx, size_t bytes, void** dev) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    ctx->allocations.push_back(p);
    *dev = p;
    return DNNMG_OK;
}

size_t field_elem(int precision) { return precision == DNNMG_FP64 ? sizeof(double) : sizeof(float); }

bool is_fp64(const dnnmg_ctx* c) { return c->precision == DNNMG_FP64; }

// Fields of [n][4] values are read and written 4 values at a time (16 bytes
// in float, 32 in double) and rows of X in 16-byte pieces; d and Y are read
// by the element.  Pointers that break this are refused before any launch.
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
bool node_fields_aligned(const dnnmg_ctx* c, std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (p && !aligned(p, 4 * field_elem(c->precision))) return false;
    return true;
}
bool elem_aligned(const dnnmg_ctx* c, std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (p && !aligned(p, field_elem(c->precision))) return false;
    return true;
}

// Wait for the context's stream, then report an expired bounded wait of
// this context's tensor-core kernels (and clear it) as ETIMEOUT.
dnnmg_status sync_and_check(dnnmg_ctx* ctx) {
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    int code = 0;
    CK(ctx, read_tc_error(ctx->tc_err, ctx->stream, &code));
    if (code)
        return fail(ctx, DNNMG_ETIMEOUT,
                    "tensor-core kernel: a bounded wait expired (code " + std::to_string(code) + ")");
    return DNNMG_OK;
}

// network inputs per patch: 2 x nodes x 4 values + the geometry features;
// the row stride of X; outputs per patch (3 per node)
int n_in(const HostHierarchy& h) { return 8 * h.npn + h.n_geo; }
int n_in_pad(const HostHierarchy& h) { return h.J == 2 ? kNInPadJ2 : kNInPad; }
int n_out(const HostHierarchy& h) { return 3 * h.npn; }
int n_in(const dnnmg_ctx* c) { return n_in(c->host); }
int n_in_pad(const dnnmg_ctx* c) { return n_in_pad(c->host); }
int n_out(const dnnmg_ctx* c) { return n_out(c->host); }

void fill_sizes(const HostHierarchy& h, int32_t precision, dnnmg_sizes* out) {
    out->n_coarse_vertices = h.nv;
    out->n_patches = h.nc;
    out->n_fine_nodes = h.n_fine;
    out->n_coarse_edges = h.ne;
    out->n_coarse_faces = h.nf;
    out->n_in = n_in(h);
    out->n_in_padded = n_in_pad(h);
    out->n_out = n_out(h);
    out->precision = precision;
    out->n_coarse_nodes = h.element == 2 ? h.n_mid : h.nv;
    out->element = h.element;
    out->reserved = 0;
}

// rows of x_coarse / b_coarse: coarse vertices (Q1) or level L+1 nodes (Q2)
int64_t coarse_nodes(const HostHierarchy& h) { return h.element == 2 ? h.n_mid : h.nv; }
bool is_q2(const dnnmg_ctx* c) { return c->host.element == 2; }

// one item of a host hierarchy into a caller buffer of `bytes` bytes
dnnmg_status copy_mesh_item(const HostHierarchy& h, int32_t item, void* host_buf, size_t bytes) {
    const void* src = nullptr;
    size_t n = 0;
    switch (item) {
        case DNNMG_PATCH_MAP: src = h.patch_map.data(); n = h.patch_map.size() * 4; break;
        case DNNMG_VALENCE: src = h.valence.data(); n = h.valence.size() * 4; break;
        case DNNMG_FINE_KIND: src = h.kind_f.data(); n = h.kind_f.size() * 4; break;
        case DNNMG_FINE_XYZ: src = h.xyz_f.data(); n = h.xyz_f.size() * 8; break;
        case DNNMG_EDGE_LENGTHS: {   // the first 12 of each patch's geometry features
            n = size_t(h.nc) * 12 * 8;
            if (bytes < n) return DNNMG_EINVAL;
            double* dst = static_cast<double*>(host_buf);
            for (int64_t c = 0; c < h.nc; ++c)
                std::memcpy(dst + 12 * c, h.geo.data() + size_t(h.n_geo) * size_t(c), 12 * 8);
            return DNNMG_OK;
        }
        case DNNMG_GEOMETRY: src = h.geo.data(); n = h.geo.size() * 8; break;
        case DNNMG_COARSE_XYZ:
            src = h.element == 2 ? h.xyz_mid.data() : h.xyz_c.data();
            n = (h.element == 2 ? h.xyz_mid.size() : h.xyz_c.size()) * 8;
            break;
        case DNNMG_COARSE_KIND:
            src = h.element == 2 ? h.kind_mid.data() : h.bc_c.data();
            n = (h.element == 2 ? h.kind_mid.size() : h.bc_c.size()) * 4;
            break;
        default: return DNNMG_EINVAL;
    }
    if (bytes < n) return DNNMG_EINVAL;
    std::memcpy(host_buf, src, n);
    return DNNMG_OK;
}

}  // namespace

extern "C" {

const char* dnnmg_strerror(dnnmg_status s) {
    const int i = -int(s);
    if (i < 0 || i >= int(sizeof(kStatusText) / sizeof(kStatusText[0]))) return "unknown status";
    return kStatusText[i];
}

const char* dnnmg_last_error(const dnnmg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int64_t dnnmg_launch_count(const dnnmg_ctx* ctx) { return ctx ? ctx->launches : 0; }

void dnnmg_destroy(dnnmg_ctx* ctx) {
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
        cudaEventDestroy(ctx->ev_ready);
        cudaEventDestroy(ctx->ev_input);
    }
    for (void* p : ctx->allocations) cudaFree(p);
    for (auto*& L : ctx->level) {
        destroy_level(L);
        L = nullptr;
    }
    cudaSetDevice(cur);
    delete ctx;
}

dnnmg_status dnnmg_create(const dnnmg_mesh_desc* mesh, const dnnmg_params* params, void* cuda_stream,
                          dnnmg_ctx** out) {
    Range nvtx_range("dnnmg_create");
    if (!out) return DNNMG_EINVAL;
    *out = nullptr;
    if (!mesh || !params) return DNNMG_EINVAL;
    if (params->features != 0 && params->features != 12 && params->features != 24) return DNNMG_EINVAL;
    if (params->patch_levels < 0 || params->patch_levels > 2 || params->element < 0 || params->element > 2)
        return DNNMG_EINVAL;
    const bool q2 = params->element == 2;
    if (q2 && params->patch_levels == 1) return DNNMG_EINVAL;   // Q2 patches have the J = 2 layout
    const int J = (params->patch_levels == 2 || q2) ? 2 : 1;
    if (params->precision < DNNMG_FP64 || params->precision > DNNMG_BF16 ||
        !(params->dt > 0.0) || !(params->nu >= 0.0) || !(params->theta >= 0.0 && params->theta <= 1.0))
        return DNNMG_EINVAL;
    dnnmg_ctx* ctx = new (std::nothrow) dnnmg_ctx();
    if (!ctx) return DNNMG_ENOMEM;
    std::string err;
    dnnmg_status st = build_hierarchy(mesh, params->features == 24 ? 24 : 12, J, &ctx->host, &err);
    if (st != DNNMG_OK) {
        delete ctx;
        return st;
    }
    ctx->host.element = q2 ? 2 : 1;
    ctx->precision = params->precision;
    ctx->op = OpParams{1.0 / params->dt, params->theta, params->nu};
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return DNNMG_ECUDA;
    }
    const HostHierarchy& h = ctx->host;
    DeviceMesh& dm = ctx->dm;
    dm.nv = h.nv;
    dm.nc = h.nc;
    dm.n_fine = h.n_fine;
    dm.n_geo = h.n_geo;
    dm.J = h.J;
    auto done = [&](dnnmg_status s) {
        if (s != DNNMG_OK) {
            dnnmg_destroy(ctx);
            return s;
        }
        *out = ctx;
        return DNNMG_OK;
    };
    int32_t* p;
#define UP(vec, field)                                                           \
    do {                                                                         \
        st = upload(ctx, vec.data(), vec.size(), &p);                            \
        if (st != DNNMG_OK) return done(st);                                     \
        dm.field = p;                                                            \
    } while (0)
    UP(h.cells, cells);
    UP(h.patch_map, patch_map);
    UP(h.node_ptr, node_ptr);
    UP(h.node_idx, node_idx);
    UP(h.vert_ptr, vert_ptr);
    UP(h.vert_idx, vert_idx);
#undef UP
    std::vector<uint8_t> fd(size_t(h.n_fine)), cd(size_t(h.nv));
    for (int64_t j = 0; j < h.n_fine; ++j) fd[j] = (h.kind_f[j] == 1 || h.kind_f[j] == 2) ? 1 : 0;
    for (int64_t v = 0; v < h.nv; ++v) cd[v] = (h.bc_c[v] == 1 || h.bc_c[v] == 2) ? 1 : 0;
    uint8_t* pu;
    if ((st = upload(ctx, fd.data(), fd.size(), &pu)) != DNNMG_OK) return done(st);
    dm.fine_dir = pu;
    if ((st = upload(ctx, cd.data(), cd.size(), &pu)) != DNNMG_OK) return done(st);
    dm.coarse_dir = pu;
    if (is_fp64(ctx)) {
        double* pd;
        if ((st = upload(ctx, h.xyz_c.data(), h.xyz_c.size(), &pd)) != DNNMG_OK) return done(st);
        dm.xyz_d = pd;
        if ((st = upload(ctx, h.geo.data(), h.geo.size(), &pd)) != DNNMG_OK) return done(st);
        dm.geo_d = pd;
    } else {
        std::vector<float> xf(h.xyz_c.begin(), h.xyz_c.end()), ef(h.geo.begin(), h.geo.end());
        float* pf;
        if ((st = upload(ctx, xf.data(), xf.size(), &pf)) != DNNMG_OK) return done(st);
        dm.xyz_f = pf;
        if ((st = upload(ctx, ef.data(), ef.size(), &pf)) != DNNMG_OK) return done(st);
        dm.geo_f = pf;
    }
    if (q2) {
        // coarse Q2 nodes (level L+1) and the fine Q2 level: the 8 cells of
        // every patch (child (i, j, k) has patch nodes (2i + a, 2j + b, 2k + c))
        dm.element = 2;
        dm.n_mid = h.n_mid;
        int32_t* q;
        if ((st = upload(ctx, h.patch_map_mid.data(), h.patch_map_mid.size(), &q)) != DNNMG_OK) return done(st);
        dm.patch_map_mid = q;
        if ((st = upload(ctx, h.mid_ptr.data(), h.mid_ptr.size(), &q)) != DNNMG_OK) return done(st);
        dm.mid_ptr = q;
        if ((st = upload(ctx, h.mid_idx.data(), h.mid_idx.size(), &q)) != DNNMG_OK) return done(st);
        dm.mid_idx = q;
        std::vector<uint8_t> md(size_t(h.n_mid));
        for (int64_t j = 0; j < h.n_mid; ++j) md[j] = (h.kind_mid[j] == 1 || h.kind_mid[j] == 2) ? 1 : 0;
        if ((st = upload(ctx, md.data(), md.size(), &pu)) != DNNMG_OK) return done(st);
        dm.mid_dir = pu;
        const int64_t ncell = 8 * h.nc;
        std::vector<int32_t> cells(size_t(27 * ncell));
        for (int64_t P = 0; P < h.nc; ++P)
            for (int t = 0; t < 8; ++t)
                for (int a = 0; a < 27; ++a) {
                    const int i = t & 1, j = (t >> 1) & 1, k = (t >> 2) & 1;
                    const int iota = (2 * i + a % 3) + 5 * (2 * j + (a / 3) % 3) + 25 * (2 * k + a / 9);
                    cells[size_t(27 * (8 * P + t) + a)] = h.patch_map[size_t(125 * P + iota)];
                }
        std::vector<int32_t> cptr(size_t(h.n_fine + 1), 0), cidx(cells.size());
        for (int32_t v : cells) cptr[size_t(v) + 1]++;
        for (int64_t j = 0; j < h.n_fine; ++j) cptr[j + 1] += cptr[j];
        {
            std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
            for (size_t e = 0; e < cells.size(); ++e) cidx[size_t(fill[size_t(cells[e])]++)] = int32_t(e);
        }
        Q2Level& L = dm.q2fine;
        L.n = h.n_fine;
        L.ncell = ncell;
        if ((st = upload(ctx, cells.data(), cells.size(), &q)) != DNNMG_OK) return done(st);
        L.cells = q;
        if ((st = upload(ctx, cptr.data(), cptr.size(), &q)) != DNNMG_OK) return done(st);
        L.node_ptr = q;
        if ((st = upload(ctx, cidx.data(), cidx.size(), &q)) != DNNMG_OK) return done(st);
        L.node_idx = q;
        double* xd;
        if ((st = upload(ctx, h.xyz_f.data(), h.xyz_f.size(), &xd)) != DNNMG_OK) return done(st);
        L.xyz = xd;
        L.dir = dm.fine_dir;
    }
    const size_t fe = field_elem(ctx->precision);
    const size_t xe = ctx->precision == DNNMG_BF16 ? 2 : fe;
    const size_t nc = size_t(h.nc), nf = size_t(h.n_fine), nv = size_t(coarse_nodes(h));
    if (q2) {
        if ((st = alloc(ctx, nf * 4 * fe, &ctx->buf_xf)) != DNNMG_OK) return done(st);
        if ((st = alloc(ctx, nc * 8 * 27 * 4 * fe, &ctx->q2_local)) != DNNMG_OK) return done(st);
    }
    const size_t npn = size_t(h.npn);
    if ((st = alloc(ctx, nc * npn * 4 * fe, &ctx->partial)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nc * 8 * 4 * fe, &ctx->partial_c)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nf * 4 * fe, &ctx->buf_r)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nc * size_t(n_in_pad(ctx)) * xe, &ctx->buf_X)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nc * size_t(n_out(ctx)) * fe, &ctx->buf_Y)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nf * 3 * fe, &ctx->buf_d)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nv * 4 * fe, &ctx->buf_xc)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nf * 4 * fe, &ctx->buf_F)) != DNNMG_OK) return done(st);
    if ((st = alloc(ctx, nv * 4 * fe, &ctx->buf_bc)) != DNNMG_OK) return done(st);
    return done(DNNMG_OK);
}

dnnmg_status dnnmg_get_sizes(const dnnmg_ctx* ctx, dnnmg_sizes* out) {
    if (!ctx || !out) return DNNMG_EINVAL;
    fill_sizes(ctx->host, ctx->precision, out);
    return DNNMG_OK;
}

dnnmg_status dnnmg_get_mesh_data(const dnnmg_ctx* ctx, int32_t item, void* host_buf, size_t bytes) {
    if (!ctx || ctx->net_only || !host_buf) return DNNMG_EINVAL;
    return copy_mesh_item(ctx->host, item, host_buf, bytes);
}

// ---- the hierarchy alone, on the host -------------------------------------------
struct dnnmg_hierarchy {
    HostHierarchy host;
};

dnnmg_status dnnmg_hierarchy_build(const dnnmg_mesh_desc* mesh, int32_t features, int32_t patch_levels,
                                   dnnmg_hierarchy** out) {
    if (!out) return DNNMG_EINVAL;
    *out = nullptr;
    if (!mesh || (features != 0 && features != 12 && features != 24) || patch_levels < 0 || patch_levels > 2)
        return DNNMG_EINVAL;
    dnnmg_hierarchy* h = new (std::nothrow) dnnmg_hierarchy();
    if (!h) return DNNMG_ENOMEM;
    std::string err;
    const dnnmg_status st = build_hierarchy(mesh, features == 24 ? 24 : 12, patch_levels == 2 ? 2 : 1, &h->host, &err);
    if (st != DNNMG_OK) {
        delete h;
        return st;
    }
    *out = h;
    return DNNMG_OK;
}

dnnmg_status dnnmg_hierarchy_sizes(const dnnmg_hierarchy* h, dnnmg_sizes* out) {
    if (!h || !out) return DNNMG_EINVAL;
    fill_sizes(h->host, -1, out);
    return DNNMG_OK;
}

dnnmg_status dnnmg_hierarchy_data(const dnnmg_hierarchy* h, int32_t item, void* host_buf, size_t bytes) {
    if (!h || !host_buf) return DNNMG_EINVAL;
    return copy_mesh_item(h->host, item, host_buf, bytes);
}

void dnnmg_hierarchy_destroy(dnnmg_hierarchy* h) { delete h; }

dnnmg_status dnnmg_set_stream(dnnmg_ctx* ctx, void* cuda_stream) {
    if (!ctx) return DNNMG_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return DNNMG_OK;
}

dnnmg_status dnnmg_set_network(dnnmg_ctx* ctx, const dnnmg_net_desc* net, const double* const* W,
                               const double* const* scale, const double* const* shift) {
    Range nvtx_range("dnnmg_set_network");
    if (!ctx || !net || !W || !net->widths || net->n_layers < 1 || net->n_layers > 64) return DNNMG_EINVAL;
    const int L = net->n_layers;
    if (net->widths[0] != n_in(ctx) || net->widths[L] != n_out(ctx))
        return fail(ctx, DNNMG_EINVAL, "network widths must start at n_in and end at n_out of the context");
    for (int i = 1; i < L; ++i) {
        const int w = net->widths[i];
        if (w < 1 || w > 4096) return fail(ctx, DNNMG_EINVAL, "hidden widths must be in [1, 4096]");
    }
    for (int i = 0; i < L; ++i)
        if (!W[i]) return DNNMG_EINVAL;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    // release a previous network's memory
    auto drop = [&](void* p) {
        if (!p) return;
        for (auto& a : ctx->allocations)
            if (a == p) {
                cudaFree(a);
                a = nullptr;
            }
    };
    for (void* p : ctx->W) drop(p);
    for (void* p : ctx->scale) drop(p);
    for (void* p : ctx->shift) drop(p);
    drop(ctx->act[0]);
    drop(ctx->act[1]);
    ctx->W.clear();
    ctx->scale.clear();
    ctx->shift.clear();
    ctx->has_net = false;
    if (!ctx->tc_err) {
        void* p = nullptr;
        dnnmg_status sa = alloc(ctx, sizeof(int), &p);
        if (sa != DNNMG_OK) return sa;
        CK(ctx, cudaMemset(p, 0, sizeof(int)));
        ctx->tc_err = static_cast<int*>(p);
    }
    ctx->n_layers = L;
    ctx->skip = net->skip;
    ctx->widths.assign(net->widths, net->widths + L + 1);
    ctx->kpad.resize(L);
    ctx->npad.resize(L);
    int maxw = 16;
    for (int i = 0; i < L; ++i) {
        const bool bf16 = ctx->precision == DNNMG_BF16;
        // tensor-core layers read K in blocks of 64 and the last layer's W
        // as a 96-row tile, SIMT layers K in steps of 16; padding is zero
        ctx->kpad[i] = i == 0 ? n_in_pad(ctx) : (bf16 ? (ctx->widths[i] + 63) / 64 * 64 : (ctx->widths[i] + 15) / 16 * 16);
        ctx->npad[i] = (bf16 && i == L - 1) ? std::max(96, ctx->widths[i + 1]) : ctx->widths[i + 1];
        if (i < L - 1) maxw = std::max(maxw, ctx->widths[i + 1]);
    }
    maxw = ctx->precision == DNNMG_BF16 ? (maxw + 63) / 64 * 64 : (maxw + 15) / 16 * 16;
    dnnmg_status st;
    for (int i = 0; i < L; ++i) {
        const int N = ctx->npad[i], K = ctx->kpad[i], n_true = ctx->widths[i + 1], k_true = ctx->widths[i];
        std::vector<double> w(size_t(N) * K, 0.0), s(size_t(N), 0.0), t(size_t(N), 0.0);
        for (int n = 0; n < n_true; ++n) {
            for (int k = 0; k < k_true; ++k) w[size_t(n) * K + k] = W[i][size_t(n) * k_true + k];
            s[n] = scale && scale[i] ? scale[i][n] : 1.0;
            t[n] = shift && shift[i] ? shift[i][n] : 0.0;
        }
        void* dw;
        void* ds;
        void* dt;
        if (ctx->precision == DNNMG_FP64) {
            double* p = nullptr;
            if ((st = upload(ctx, w.data(), w.size(), &p)) != DNNMG_OK) return st;
            dw = p;
            if ((st = upload(ctx, s.data(), s.size(), &p)) != DNNMG_OK) return st;
            ds = p;
            if ((st = upload(ctx, t.data(), t.size(), &p)) != DNNMG_OK) return st;
            dt = p;
        } else {
            std::vector<float> sf(s.begin(), s.end()), tf(t.begin(), t.end());
            float* p = nullptr;
            if (ctx->precision == DNNMG_FP32) {
                std::vector<float> wf(w.begin(), w.end());
                if ((st = upload(ctx, wf.data(), wf.size(), &p)) != DNNMG_OK) return st;
                dw = p;
            } else {
                std::vector<__nv_bfloat16> wb(w.size());
                for (size_t e = 0; e < w.size(); ++e) wb[e] = __float2bfloat16_rn(float(w[e]));
                __nv_bfloat16* pb = nullptr;
                if ((st = upload(ctx, wb.data(), wb.size(), &pb)) != DNNMG_OK) return st;
                dw = pb;
            }
            if ((st = upload(ctx, sf.data(), sf.size(), &p)) != DNNMG_OK) return st;
            ds = p;
            if ((st = upload(ctx, tf.data(), tf.size(), &p)) != DNNMG_OK) return st;
            dt = p;
        }
        ctx->W.push_back(dw);
        ctx->scale.push_back(ds);
        ctx->shift.push_back(dt);
    }
    ctx->act_rows = ctx->net_capacity > 0 ? ctx->net_capacity : std::max<int64_t>(ctx->host.nc, 1);
    ctx->act_ld = maxw;
    const size_t ae = ctx->precision == DNNMG_FP64 ? 8 : (ctx->precision == DNNMG_FP32 ? 4 : 2);
    for (int b = 0; b < 2; ++b) {
        if ((st = alloc(ctx, size_t(ctx->act_rows) * maxw * ae, &ctx->act[b])) != DNNMG_OK) return st;
        // columns beyond a layer's width are never written and must read as 0
        CK(ctx, cudaMemset(ctx->act[b], 0, size_t(ctx->act_rows) * maxw * ae));
    }
    ctx->has_net = true;
    return DNNMG_OK;
}

}  // extern "C"

namespace {

// The Q2 stages (J = 2 layout): x~ = P x^L into the context's buffer, the
// fine cells' rows, their gather; the rhs at x~ + d and its restriction.
constexpr double kQ2Alpha0 = 0.02, kQ2Delta0 = 0.1;   // Eq. (8) parameters of the fine level

template <typename T>
cudaError_t q2_residual(dnnmg_ctx* ctx, const T* xc, const T* F, T* r, cudaEvent_t F_ready) {
    const DeviceMesh& dm = ctx->dm;
    cudaError_t e = q2_prolongate<T>(dm, xc, static_cast<T*>(ctx->buf_xf), ctx->stream);
    if (e == cudaSuccess)
        e = q2_level_local<T>(dm.q2fine, 0, static_cast<const T*>(ctx->buf_xf), nullptr, ctx->op, kQ2Alpha0,
                              kQ2Delta0, 1, static_cast<T*>(ctx->q2_local), ctx->stream);
    if (e == cudaSuccess && F_ready) e = cudaStreamWaitEvent(ctx->stream, F_ready, 0);
    if (e == cudaSuccess) e = q2_gather<T>(dm.q2fine, 0, static_cast<const T*>(ctx->q2_local), F, r, ctx->stream);
    ctx->launches += 3;
    return e;
}

template <typename T>
cudaError_t q2_rhs_restrict(dnnmg_ctx* ctx, const T* xc, const T* d, T* b_fine, T* b_coarse) {
    const DeviceMesh& dm = ctx->dm;
    T* xf = static_cast<T*>(ctx->buf_xf);
    cudaError_t e = q2_prolongate<T>(dm, xc, xf, ctx->stream);
    if (e == cudaSuccess)
        e = q2_level_local<T>(dm.q2fine, 1, xf, d, ctx->op, kQ2Alpha0, kQ2Delta0, 0, static_cast<T*>(ctx->q2_local),
                              ctx->stream);
    // without b_fine the prolongated field's buffer (read above) holds it
    T* bf = b_fine ? b_fine : xf;
    if (e == cudaSuccess) e = q2_gather<T>(dm.q2fine, 1, static_cast<const T*>(ctx->q2_local), nullptr, bf, ctx->stream);
    ctx->launches += 3;
    if (e == cudaSuccess && b_coarse) {
        e = q2_restrict<T>(dm, bf, static_cast<T*>(ctx->partial), b_coarse, ctx->stream);
        ctx->launches += 2;
    }
    return e;
}

template <typename T, typename TX>
cudaError_t q2_local_restrict_step(dnnmg_ctx* ctx, const T* xc, const T* r, TX* X) {
    const DeviceMesh& dm = ctx->dm;
    T* xf = static_cast<T*>(ctx->buf_xf);
    cudaError_t e = q2_prolongate<T>(dm, xc, xf, ctx->stream);
    const T* geo = sizeof(T) == 8 ? reinterpret_cast<const T*>(dm.geo_d) : reinterpret_cast<const T*>(dm.geo_f);
    if (e == cudaSuccess) e = q2_local_restrict<T, TX>(dm, xf, r, geo, kNInPadJ2, X, ctx->stream);
    ctx->launches += 2;
    return e;
}

}  // namespace

extern "C" {

dnnmg_status dnnmg_prolongate(dnnmg_ctx* ctx, const void* x_coarse_dev, void* x_fine_dev) {
    Range nvtx_range("dnnmg_prolongate");
    if (!ctx || ctx->net_only || !x_coarse_dev || !x_fine_dev) return DNNMG_EINVAL;
    if (!node_fields_aligned(ctx, {x_coarse_dev, x_fine_dev})) return fail(ctx, DNNMG_EINVAL, "misaligned field");
    cudaError_t e;
    if (is_q2(ctx))
        e = is_fp64(ctx) ? q2_prolongate(ctx->dm, (const double*)x_coarse_dev, (double*)x_fine_dev, ctx->stream)
                         : q2_prolongate(ctx->dm, (const float*)x_coarse_dev, (float*)x_fine_dev, ctx->stream);
    else
        e = is_fp64(ctx) ? launch_prolongate(ctx->dm, (const double*)x_coarse_dev, (double*)x_fine_dev, ctx->stream)
                         : launch_prolongate(ctx->dm, (const float*)x_coarse_dev, (float*)x_fine_dev, ctx->stream);
    ctx->launches += 1;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "prolongate");
    return DNNMG_OK;
}

dnnmg_status dnnmg_patch_targets(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* v_fine_dev, float* T_dev,
                                 int64_t ldt) {
    Range nvtx_range("dnnmg_patch_targets");
    if (!ctx || ctx->net_only || !x_coarse_dev || !v_fine_dev || !T_dev) return DNNMG_EINVAL;
    if (ldt < n_out(ctx)) return fail(ctx, DNNMG_EINVAL, "ldt < n_out");
    if (!node_fields_aligned(ctx, {x_coarse_dev, v_fine_dev})) return fail(ctx, DNNMG_EINVAL, "misaligned field");
    if (!ctx->buf_xf) {
        const size_t bytes = size_t(ctx->host.n_fine) * 4 * field_elem(ctx->precision);
        const dnnmg_status st = alloc(ctx, bytes, &ctx->buf_xf);
        if (st != DNNMG_OK) return st;
    }
    const int npn = ctx->host.npn;
    cudaError_t e;
    if (is_fp64(ctx)) {
        const double* xc = static_cast<const double*>(x_coarse_dev);
        double* xt = static_cast<double*>(ctx->buf_xf);
        e = is_q2(ctx) ? q2_prolongate(ctx->dm, xc, xt, ctx->stream) : launch_prolongate(ctx->dm, xc, xt, ctx->stream);
        if (e == cudaSuccess)
            e = launch_targets(ctx->dm, npn, static_cast<const double*>(v_fine_dev), xt, T_dev, ldt, ctx->stream);
    } else {
        const float* xc = static_cast<const float*>(x_coarse_dev);
        float* xt = static_cast<float*>(ctx->buf_xf);
        e = is_q2(ctx) ? q2_prolongate(ctx->dm, xc, xt, ctx->stream) : launch_prolongate(ctx->dm, xc, xt, ctx->stream);
        if (e == cudaSuccess)
            e = launch_targets(ctx->dm, npn, static_cast<const float*>(v_fine_dev), xt, T_dev, ldt, ctx->stream);
    }
    ctx->launches += 2;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "patch targets");
    return DNNMG_OK;
}

// the residual; the gather reading F waits for F_ready when given
static dnnmg_status residual_impl(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* F_dev, void* r_dev,
                           cudaEvent_t F_ready) {
    if (is_q2(ctx)) {
        cudaError_t e = is_fp64(ctx) ? q2_residual(ctx, (const double*)x_coarse_dev, (const double*)F_dev,
                                                   (double*)r_dev, F_ready)
                                     : q2_residual(ctx, (const float*)x_coarse_dev, (const float*)F_dev,
                                                   (float*)r_dev, F_ready);
        return e == cudaSuccess ? DNNMG_OK : cuda_fail(ctx, e, "residual (Q2)");
    }
    int launches = 0;
    cudaError_t e = is_fp64(ctx)
                        ? launch_residual(ctx->dm, ctx->op, (const double*)x_coarse_dev, (const double*)F_dev,
                                          (double*)r_dev, (double*)ctx->partial, ctx->stream, &launches, F_ready)
                        : launch_residual(ctx->dm, ctx->op, (const float*)x_coarse_dev, (const float*)F_dev,
                                          (float*)r_dev, (float*)ctx->partial, ctx->stream, &launches, F_ready);
    ctx->launches += launches;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "residual");
    return DNNMG_OK;
}

dnnmg_status dnnmg_residual(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* F_dev, void* r_dev) {
    Range nvtx_range("dnnmg_residual");
    if (!ctx || ctx->net_only || !x_coarse_dev || !F_dev || !r_dev) return DNNMG_EINVAL;
    if (!node_fields_aligned(ctx, {x_coarse_dev, F_dev, r_dev})) return fail(ctx, DNNMG_EINVAL, "misaligned field");
    return residual_impl(ctx, x_coarse_dev, F_dev, r_dev, nullptr);
}


dnnmg_status dnnmg_local_restrict(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* r_dev, void* X_dev) {
    Range nvtx_range("dnnmg_local_restrict");
    if (!ctx || ctx->net_only || !x_coarse_dev || !r_dev || !X_dev) return DNNMG_EINVAL;
    if (!node_fields_aligned(ctx, {x_coarse_dev, r_dev}) || !aligned(X_dev, 16))
        return fail(ctx, DNNMG_EINVAL, "misaligned field");
    cudaError_t e;
    if (is_q2(ctx)) {
        if (ctx->precision == DNNMG_FP64)
            e = q2_local_restrict_step(ctx, (const double*)x_coarse_dev, (const double*)r_dev, (double*)X_dev);
        else if (ctx->precision == DNNMG_FP32)
            e = q2_local_restrict_step(ctx, (const float*)x_coarse_dev, (const float*)r_dev, (float*)X_dev);
        else
            e = q2_local_restrict_step(ctx, (const float*)x_coarse_dev, (const float*)r_dev, (__nv_bfloat16*)X_dev);
        return e == cudaSuccess ? DNNMG_OK : cuda_fail(ctx, e, "local_restrict (Q2)");
    }
    if (ctx->precision == DNNMG_FP64)
        e = launch_local_restrict(ctx->dm, (const double*)x_coarse_dev, (const double*)r_dev, (double*)X_dev, ctx->stream);
    else if (ctx->precision == DNNMG_FP32)
        e = launch_local_restrict(ctx->dm, (const float*)x_coarse_dev, (const float*)r_dev, (float*)X_dev, ctx->stream);
    else
        e = launch_local_restrict(ctx->dm, (const float*)x_coarse_dev, (const float*)r_dev, (__nv_bfloat16*)X_dev,
                                  ctx->stream);
    ctx->launches += 1;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "local_restrict");
    return DNNMG_OK;
}

// The network; withhold_first_load (tensor-core form only) arms the first
// layer's first operand stage without filling it, to test the bounded waits.
static dnnmg_status network_impl(dnnmg_ctx* ctx, const void* X_dev, void* Y_dev, int64_t n_rows,
                                 int withhold_first_load) {
    if (!ctx || !X_dev || !Y_dev || n_rows < 0) return DNNMG_EINVAL;
    if (!aligned(X_dev, 16) || !elem_aligned(ctx, {Y_dev})) return fail(ctx, DNNMG_EINVAL, "misaligned field");
    if (!ctx->has_net) return fail(ctx, DNNMG_ESTATE, "dnnmg_network before dnnmg_set_network");
    if (n_rows > ctx->act_rows) return fail(ctx, DNNMG_EINVAL, "n_rows exceeds the activation capacity");
    if (ctx->wait_test_armed && ctx->precision == DNNMG_BF16) {
        withhold_first_load = 1;
        ctx->wait_test_armed = 0;
    }
    const int L = ctx->n_layers;
    for (int i = 0; i < L; ++i) {
        const bool last = i == L - 1;
        const void* A = i == 0 ? X_dev : ctx->act[(i - 1) & 1];
        const int64_t lda = i == 0 ? n_in_pad(ctx) : ctx->act_ld;
        void* C = last ? Y_dev : ctx->act[i & 1];
        const int64_t ldc = last ? n_out(ctx) : ctx->act_ld;
        const bool skip = ctx->skip && i >= 1 && !last && ctx->widths[i] == ctx->widths[i + 1];
        const void* R = skip ? A : nullptr;
        const int N = ctx->npad[i], K = ctx->kpad[i];
        cudaError_t e;
        if (ctx->precision == DNNMG_FP64) {
            e = launch_layer_simt((const double*)A, lda, (const double*)ctx->W[i], K, (const double*)ctx->scale[i],
                                  (const double*)ctx->shift[i], (double*)C, ldc, (const double*)R, lda, n_rows, N, K,
                                  !last, ctx->stream);
        } else if (ctx->precision == DNNMG_FP32) {
            e = launch_layer_simt((const float*)A, lda, (const float*)ctx->W[i], K, (const float*)ctx->scale[i],
                                  (const float*)ctx->shift[i], (float*)C, ldc, (const float*)R, lda, n_rows, N, K,
                                  !last, ctx->stream);
        } else {
            e = launch_layer_tc((const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)ctx->W[i], K, N,
                                (const float*)ctx->scale[i], (const float*)ctx->shift[i], C, ldc, !last,
                                (const __nv_bfloat16*)R, lda, n_rows, ctx->widths[i + 1], K, !last, ctx->stream,
                                ctx->tc_err, i == 0 ? withhold_first_load : 0);
        }
        ctx->launches += 1;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "network layer");
    }
    return DNNMG_OK;
}

dnnmg_status dnnmg_network(dnnmg_ctx* ctx, const void* X_dev, void* Y_dev, int64_t n_rows) {
    Range nvtx_range("dnnmg_network");
    return network_impl(ctx, X_dev, Y_dev, n_rows, 0);
}

dnnmg_status dnnmg_network_wait_test(dnnmg_ctx* ctx, const void* X_dev, void* Y_dev, int64_t n_rows) {
    if (!ctx || ctx->precision != DNNMG_BF16) return DNNMG_EUNSUPPORTED;
    Range nvtx_range("dnnmg_network_wait_test");
    return network_impl(ctx, X_dev, Y_dev, n_rows, 1);
}

dnnmg_status dnnmg_arm_wait_test(dnnmg_ctx* ctx) {
    if (!ctx || ctx->precision != DNNMG_BF16) return DNNMG_EUNSUPPORTED;
    ctx->wait_test_armed = 1;
    return DNNMG_OK;
}

dnnmg_status dnnmg_extend(dnnmg_ctx* ctx, const void* Y_dev, void* d_dev) {
    Range nvtx_range("dnnmg_extend");
    if (!ctx || ctx->net_only || !Y_dev || !d_dev) return DNNMG_EINVAL;
    if (!elem_aligned(ctx, {Y_dev, d_dev})) return fail(ctx, DNNMG_EINVAL, "misaligned field");
    cudaError_t e = is_fp64(ctx) ? launch_extend(ctx->dm, (const double*)Y_dev, (double*)d_dev, ctx->stream)
                                 : launch_extend(ctx->dm, (const float*)Y_dev, (float*)d_dev, ctx->stream);
    ctx->launches += 1;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "extend");
    return DNNMG_OK;
}

dnnmg_status dnnmg_rhs_restrict(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* d_dev, void* b_fine_dev,
                                void* b_coarse_dev) {
    Range nvtx_range("dnnmg_rhs_restrict");
    if (!ctx || ctx->net_only || !x_coarse_dev || !d_dev) return DNNMG_EINVAL;
    if (!node_fields_aligned(ctx, {x_coarse_dev, b_fine_dev, b_coarse_dev}) || !elem_aligned(ctx, {d_dev}))
        return fail(ctx, DNNMG_EINVAL, "misaligned field");
    if (is_q2(ctx)) {
        cudaError_t e = is_fp64(ctx) ? q2_rhs_restrict(ctx, (const double*)x_coarse_dev, (const double*)d_dev,
                                                       (double*)b_fine_dev, (double*)b_coarse_dev)
                                     : q2_rhs_restrict(ctx, (const float*)x_coarse_dev, (const float*)d_dev,
                                                       (float*)b_fine_dev, (float*)b_coarse_dev);
        return e == cudaSuccess ? DNNMG_OK : cuda_fail(ctx, e, "rhs_restrict (Q2)");
    }
    int launches = 0;
    cudaError_t e =
        is_fp64(ctx)
            ? launch_rhs_restrict(ctx->dm, ctx->op, (const double*)x_coarse_dev, (const double*)d_dev,
                                  (double*)b_fine_dev, (double*)b_coarse_dev, (double*)ctx->partial,
                                  (double*)ctx->partial_c, ctx->stream, &launches)
            : launch_rhs_restrict(ctx->dm, ctx->op, (const float*)x_coarse_dev, (const float*)d_dev,
                                  (float*)b_fine_dev, (float*)b_coarse_dev, (float*)ctx->partial,
                                  (float*)ctx->partial_c, ctx->stream, &launches);
    ctx->launches += launches;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rhs_restrict");
    return DNNMG_OK;
}

dnnmg_status dnnmg_restrict(dnnmg_ctx* ctx, const void* b_fine_dev, void* b_coarse_dev) {
    Range nvtx_range("dnnmg_restrict");
    if (!ctx || ctx->net_only || !b_fine_dev || !b_coarse_dev) return DNNMG_EINVAL;
    if (!node_fields_aligned(ctx, {b_fine_dev, b_coarse_dev})) return fail(ctx, DNNMG_EINVAL, "misaligned field");
    if (is_q2(ctx)) {
        cudaError_t e = is_fp64(ctx) ? q2_restrict(ctx->dm, (const double*)b_fine_dev, (double*)ctx->partial,
                                                   (double*)b_coarse_dev, ctx->stream)
                                     : q2_restrict(ctx->dm, (const float*)b_fine_dev, (float*)ctx->partial,
                                                   (float*)b_coarse_dev, ctx->stream);
        ctx->launches += 2;
        return e == cudaSuccess ? DNNMG_OK : cuda_fail(ctx, e, "restrict (Q2)");
    }
    cudaError_t e = is_fp64(ctx) ? launch_restrict(ctx->dm, (const double*)b_fine_dev, (double*)b_coarse_dev,
                                                   (double*)ctx->partial_c, ctx->stream)
                                 : launch_restrict(ctx->dm, (const float*)b_fine_dev, (float*)b_coarse_dev,
                                                   (float*)ctx->partial_c, ctx->stream);
    ctx->launches += 2;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "restrict");
    return DNNMG_OK;
}

dnnmg_status dnnmg_patch_step(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* F_dev, void* b_fine_dev,
                              void* b_coarse_dev) {
    Range nvtx_range("dnnmg_patch_step");
    if (!ctx || ctx->net_only || !x_coarse_dev || !F_dev) return DNNMG_EINVAL;
    if (!ctx->has_net) return fail(ctx, DNNMG_ESTATE, "dnnmg_patch_step before dnnmg_set_network");
    dnnmg_status st;
    if ((st = dnnmg_residual(ctx, x_coarse_dev, F_dev, ctx->buf_r)) != DNNMG_OK) return st;
    if ((st = dnnmg_local_restrict(ctx, x_coarse_dev, ctx->buf_r, ctx->buf_X)) != DNNMG_OK) return st;
    if ((st = dnnmg_network(ctx, ctx->buf_X, ctx->buf_Y, ctx->host.nc)) != DNNMG_OK) return st;
    if ((st = dnnmg_extend(ctx, ctx->buf_Y, ctx->buf_d)) != DNNMG_OK) return st;
    return dnnmg_rhs_restrict(ctx, x_coarse_dev, ctx->buf_d, b_fine_dev, b_coarse_dev);
}

dnnmg_status dnnmg_patch_step_host(dnnmg_ctx* ctx, const void* x_coarse_host, const void* F_host,
                                   void* b_fine_host, void* b_coarse_host) {
    Range nvtx_range("dnnmg_patch_step_host");
    if (!ctx || ctx->net_only || !x_coarse_host || !F_host) return DNNMG_EINVAL;
    if (!ctx->has_net) return fail(ctx, DNNMG_ESTATE, "dnnmg_patch_step_host before dnnmg_set_network");
    const size_t fe = field_elem(ctx->precision);
    const size_t nv = size_t(coarse_nodes(ctx->host)), nf = size_t(ctx->host.n_fine);
    if (!ctx->copy_stream) {
        CK(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        CK(ctx, cudaEventCreateWithFlags(&ctx->ev_ready, cudaEventDisableTiming));
        CK(ctx, cudaEventCreateWithFlags(&ctx->ev_input, cudaEventDisableTiming));
    }
    // x^L on the context's stream; F (the large input) on the copy stream,
    // after everything already queued on the context's stream, while the
    // element kernel of the residual (which needs only x^L) runs
    CK(ctx, cudaEventRecord(ctx->ev_ready, ctx->stream));
    CK(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_ready, 0));
    // from the first copy on, an error return first waits for both streams,
    // so that no copy still reads the caller's host buffers afterwards
    auto drain = [&](dnnmg_status st) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamSynchronize(ctx->stream);
        return st;
    };
    cudaError_t ce = cudaMemcpyAsync(ctx->buf_xc, x_coarse_host, nv * 4 * fe, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(ctx->buf_F, F_host, nf * 4 * fe, cudaMemcpyHostToDevice, ctx->copy_stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(ctx->ev_input, ctx->copy_stream);
    if (ce != cudaSuccess) return drain(cuda_fail(ctx, ce, "input upload"));
    dnnmg_status st;
    if ((st = residual_impl(ctx, ctx->buf_xc, ctx->buf_F, ctx->buf_r, ctx->ev_input)) != DNNMG_OK) return drain(st);
    if ((st = dnnmg_local_restrict(ctx, ctx->buf_xc, ctx->buf_r, ctx->buf_X)) != DNNMG_OK) return drain(st);
    if ((st = dnnmg_network(ctx, ctx->buf_X, ctx->buf_Y, ctx->host.nc)) != DNNMG_OK) return drain(st);
    if ((st = dnnmg_extend(ctx, ctx->buf_Y, ctx->buf_d)) != DNNMG_OK) return drain(st);
    if ((st = dnnmg_rhs_restrict(ctx, ctx->buf_xc, ctx->buf_d, ctx->buf_F, ctx->buf_bc)) != DNNMG_OK) return drain(st);
    if (b_fine_host) ce = cudaMemcpyAsync(b_fine_host, ctx->buf_F, nf * 4 * fe, cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess && b_coarse_host)
        ce = cudaMemcpyAsync(b_coarse_host, ctx->buf_bc, nv * 4 * fe, cudaMemcpyDeviceToHost, ctx->stream);
    if (ce != cudaSuccess) return drain(cuda_fail(ctx, ce, "output download"));
    return drain(sync_and_check(ctx));
}

dnnmg_status dnnmg_get_buffer(dnnmg_ctx* ctx, int32_t which, void** dev_ptr) {
    if (!ctx || !dev_ptr) return DNNMG_EINVAL;
    switch (which) {
        case DNNMG_BUF_R: *dev_ptr = ctx->buf_r; break;
        case DNNMG_BUF_X: *dev_ptr = ctx->buf_X; break;
        case DNNMG_BUF_Y: *dev_ptr = ctx->buf_Y; break;
        case DNNMG_BUF_D: *dev_ptr = ctx->buf_d; break;
        default: return DNNMG_EINVAL;
    }
    return DNNMG_OK;
}

dnnmg_status dnnmg_sync(dnnmg_ctx* ctx, int64_t timeout_us) {
    if (!ctx) return DNNMG_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) return sync_and_check(ctx);
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "cudaStreamQuery");
        if (timeout_us >= 0) {
            const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (us > timeout_us) return fail(ctx, DNNMG_ETIMEOUT, "dnnmg_sync: timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}


// ---- Newton solver and time loop -------------------------------------------------

void dnnmg_solver_defaults(dnnmg_solver_params* p) {
    if (!p) return;
    p->alpha0 = 0.02;
    p->delta0 = 0.1;
    p->newton_atol = 1e-11;
    p->newton_rtol = 1e-12;
    p->newton_max = 25;
    p->gmres_restart = 40;
    p->gmres_max = 400;
    p->mg_levels = 0;
    p->gmres_rtol = 1e-10;
    p->rho_max = 0.1;
    p->mg_pre = 2;
    p->mg_post = 2;
    p->mg_omega = 0.7;
    p->mg_smoother = 0;
    p->mg_bf16 = 0;
}

dnnmg_status dnnmg_hierarchy_mg(const dnnmg_hierarchy* h, int32_t level, int32_t mg_levels, int32_t max_levels,
                                int32_t* n_levels, int64_t* nodes) {
    if (!h || !n_levels || (level != DNNMG_LEVEL_COARSE && level != DNNMG_LEVEL_FINE) || mg_levels < 0 ||
        max_levels < 0 || (max_levels > 0 && !nodes))
        return DNNMG_EINVAL;
    std::vector<HostLevel> lv(1);
    build_level(h->host, level == DNNMG_LEVEL_FINE, &lv[0]);
    for (int k = 0; k < mg_levels; ++k) {
        HostLevel c;
        MgTransfer t;
        if (!coarsen_level(lv.back(), &c, &t)) break;
        lv.push_back(std::move(c));
    }
    *n_levels = int32_t(lv.size());
    for (int k = 0; k < max_levels && k < int(lv.size()); ++k) nodes[k] = lv[size_t(k)].n;
    return DNNMG_OK;
}

}  // extern "C"

namespace {

dnnmg_status get_level(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, DeviceLevel** out) {
    if (level != DNNMG_LEVEL_COARSE && level != DNNMG_LEVEL_FINE) return DNNMG_EINVAL;
    if (!ctx->level[level]) {
        const int krylov = prm && prm->gmres_restart > 0 ? prm->gmres_restart : 40;
        if (krylov > 200) return fail(ctx, DNNMG_EINVAL, "gmres_restart > 200");
        const int mg = prm ? prm->mg_levels : 0;
        if (mg < 0 || mg > 16) return fail(ctx, DNNMG_EINVAL, "mg_levels outside [0, 16]");
        cudaError_t e = create_level(ctx->host, level == DNNMG_LEVEL_FINE, krylov, mg, &ctx->level[level]);
        if (e == cudaErrorInvalidValue)
            return fail(ctx, DNNMG_EINVAL, "the coarsest multigrid level is too large for the dense solve "
                                           "(more than 8192 unknowns): allow more levels");
        if (e != cudaSuccess) return cuda_fail(ctx, e, "create_level");
    }
    *out = ctx->level[level];
    return DNNMG_OK;
}

__global__ void to_float_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = float(a[i]);
}
__global__ void to_double_kernel(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = double(a[i]);
}

}  // namespace

extern "C" {

dnnmg_status dnnmg_level_info(dnnmg_ctx* ctx, int32_t level, int64_t* n_nodes, int32_t* grouped) {
    if (!ctx) return DNNMG_EINVAL;
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, nullptr, &L);
    if (st != DNNMG_OK) return st;
    if (n_nodes) *n_nodes = level_nodes(L);
    if (grouped) *grouped = level_lps(L) ? 1 : 0;
    return DNNMG_OK;
}

dnnmg_status dnnmg_level_operator(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, const double* x_dev,
                                  double* Ax_dev) {
    if (!ctx || ctx->net_only || !x_dev || !Ax_dev) return DNNMG_EINVAL;
    dnnmg_solver_params d;
    dnnmg_solver_defaults(&d);
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, prm, &L);
    if (st != DNNMG_OK) return st;
    CK(ctx, level_operator(L, ctx->op, prm ? prm : &d, x_dev, Ax_dev, ctx->stream));
    ctx->launches += 2;
    return DNNMG_OK;
}

dnnmg_status dnnmg_level_rhs(dnnmg_ctx* ctx, int32_t level, const double* x_old_dev, double* b_dev) {
    if (!ctx || ctx->net_only || !x_old_dev || !b_dev) return DNNMG_EINVAL;
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, nullptr, &L);
    if (st != DNNMG_OK) return st;
    CK(ctx, level_rhs(L, ctx->op, x_old_dev, b_dev, ctx->stream));
    ctx->launches += 3;
    return DNNMG_OK;
}

dnnmg_status dnnmg_level_jacobian(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, const double* x_dev,
                                  double* dense_host, size_t bytes) {
    if (!ctx || ctx->net_only || !x_dev || !dense_host) return DNNMG_EINVAL;
    dnnmg_solver_params d;
    dnnmg_solver_defaults(&d);
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, prm, &L);
    if (st != DNNMG_OK) return st;
    const int64_t N = 4 * level_nodes(L);
    if (N > 8192 || bytes < size_t(N) * size_t(N) * 8) return fail(ctx, DNNMG_EINVAL, "level too large for a dense Jacobian");
    CK(ctx, level_dense_jacobian(L, ctx->op, prm ? prm : &d, x_dev, dense_host, ctx->stream));
    return DNNMG_OK;
}

dnnmg_status dnnmg_level_mg(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, int32_t max_levels,
                            int32_t* n_levels, int64_t* nodes) {
    if (!ctx || ctx->net_only || !n_levels || max_levels < 0 || (max_levels > 0 && !nodes)) return DNNMG_EINVAL;
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, prm, &L);
    if (st != DNNMG_OK) return st;
    *n_levels = 1 + level_mg_depth(L);
    for (int k = 0; k < max_levels && k < *n_levels; ++k) nodes[k] = level_mg_nodes(L, k);
    return DNNMG_OK;
}

dnnmg_status dnnmg_solve(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, const double* b_dev,
                         double* x_dev, dnnmg_solve_stats* stats) {
    Range nvtx_range("dnnmg_solve");
    if (!ctx || ctx->net_only || !b_dev || !x_dev) return DNNMG_EINVAL;
    dnnmg_solver_params d;
    dnnmg_solver_defaults(&d);
    if (!prm) prm = &d;
    if (prm->mg_bf16 < 0 || prm->mg_bf16 > 1 || prm->mg_smoother < 0 || prm->mg_smoother > 1 || prm->newton_max < 0 || prm->gmres_max < 1 ||
        prm->mg_pre < 0 || prm->mg_post < 0 || prm->mg_pre + prm->mg_post > 64 || !(prm->mg_omega > 0.0) ||
        prm->mg_omega > 2.0)
        return DNNMG_EINVAL;
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, prm, &L);
    if (st != DNNMG_OK) return st;
    dnnmg_solve_stats s{};
    cudaError_t e = level_solve(L, ctx->op, prm, b_dev, x_dev, ctx->stream, &s);
    if (stats) *stats = s;
    if (e == cudaErrorUnknown && !std::isfinite(s.residual)) return fail(ctx, DNNMG_ENAN, "non-finite residual");
    CK(ctx, e);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return s.converged ? DNNMG_OK : fail(ctx, DNNMG_ENOCONV, "Newton tolerance not reached");
}

dnnmg_status dnnmg_time_step(dnnmg_ctx* ctx, int32_t n_steps, const dnnmg_solver_params* prm, double* x_coarse_dev,
                             double* b_coarse_dev, void* F_dev, dnnmg_solve_stats* stats) {
    Range nvtx_range("dnnmg_time_step");
    if (!ctx || ctx->net_only || !x_coarse_dev || !b_coarse_dev || !F_dev || n_steps < 0) return DNNMG_EINVAL;
    if (!ctx->has_net) return fail(ctx, DNNMG_ESTATE, "dnnmg_time_step before dnnmg_set_network");
    const int64_t nv = coarse_nodes(ctx->host);
    dnnmg_status st;
    if (!is_fp64(ctx) && !ctx->xc_field) {
        if ((st = alloc(ctx, size_t(nv) * 4 * 4, &ctx->xc_field)) != DNNMG_OK) return st;
        if ((st = alloc(ctx, size_t(nv) * 4 * 4, &ctx->bc_field)) != DNNMG_OK) return st;
    }
    for (int32_t k = 0; k < n_steps; ++k) {
        st = dnnmg_step_begin(ctx, prm, 1, x_coarse_dev, b_coarse_dev, F_dev, ctx->buf_X, stats);
        if (st != DNNMG_OK && st != DNNMG_ENOCONV) return st;
        if ((st = dnnmg_network(ctx, ctx->buf_X, ctx->buf_Y, ctx->host.nc)) != DNNMG_OK) return st;
        if ((st = dnnmg_step_end(ctx, ctx->buf_Y, F_dev, b_coarse_dev)) != DNNMG_OK) return st;
        // the next coarse solve reads b_coarse, which the network fed: stop
        // at once if one of its bounded waits expired
        if ((st = sync_and_check(ctx)) != DNNMG_OK) return st;
    }
    return sync_and_check(ctx);
}

dnnmg_status dnnmg_step_begin(dnnmg_ctx* ctx, const dnnmg_solver_params* prm, int32_t solve, double* x_coarse_dev,
                              const double* b_coarse_dev, const void* F_dev, void* X_dev, dnnmg_solve_stats* stats) {
    Range nvtx_range("dnnmg_step_begin");
    if (!ctx || ctx->net_only || !x_coarse_dev || !F_dev || !X_dev || (solve && !b_coarse_dev)) return DNNMG_EINVAL;
    const int64_t nv = coarse_nodes(ctx->host);
    dnnmg_status st = DNNMG_OK, solve_st = DNNMG_OK;
    if (!is_fp64(ctx) && !ctx->xc_field) {
        if ((st = alloc(ctx, size_t(nv) * 4 * 4, &ctx->xc_field)) != DNNMG_OK) return st;
        if ((st = alloc(ctx, size_t(nv) * 4 * 4, &ctx->bc_field)) != DNNMG_OK) return st;
    }
    if (solve) {
        solve_st = dnnmg_solve(ctx, DNNMG_LEVEL_COARSE, prm, b_coarse_dev, x_coarse_dev, stats);
        if (solve_st != DNNMG_OK && solve_st != DNNMG_ENOCONV) return solve_st;
    }
    const void* xf = x_coarse_dev;
    if (!is_fp64(ctx)) {
        to_float_kernel<<<unsigned((4 * nv + 255) / 256), 256, 0, ctx->stream>>>(4 * nv, x_coarse_dev,
                                                                                (float*)ctx->xc_field);
        CK(ctx, cudaGetLastError());
        ctx->launches += 1;
        xf = ctx->xc_field;
    }
    if ((st = dnnmg_residual(ctx, xf, F_dev, ctx->buf_r)) != DNNMG_OK) return st;
    if ((st = dnnmg_local_restrict(ctx, xf, ctx->buf_r, X_dev)) != DNNMG_OK) return st;
    ctx->last_xc = xf;
    return solve_st;
}

dnnmg_status dnnmg_step_end(dnnmg_ctx* ctx, const void* Y_dev, void* F_dev, double* b_coarse_dev) {
    Range nvtx_range("dnnmg_step_end");
    if (!ctx || ctx->net_only || !Y_dev || !F_dev || !b_coarse_dev) return DNNMG_EINVAL;
    if (!ctx->last_xc) return fail(ctx, DNNMG_ESTATE, "dnnmg_step_end before dnnmg_step_begin");
    const int64_t nv = coarse_nodes(ctx->host);
    dnnmg_status st;
    if ((st = dnnmg_extend(ctx, Y_dev, ctx->buf_d)) != DNNMG_OK) return st;
    // the coarse state of the last dnnmg_step_begin (caller's array in FP64, else its float copy)
    if (is_fp64(ctx)) return dnnmg_rhs_restrict(ctx, ctx->last_xc, ctx->buf_d, F_dev, b_coarse_dev);
    if ((st = dnnmg_rhs_restrict(ctx, ctx->last_xc, ctx->buf_d, F_dev, ctx->bc_field)) != DNNMG_OK) return st;
    to_double_kernel<<<unsigned((4 * nv + 255) / 256), 256, 0, ctx->stream>>>(4 * nv, (const float*)ctx->bc_field,
                                                                             b_coarse_dev);
    CK(ctx, cudaGetLastError());
    ctx->launches += 1;
    return DNNMG_OK;
}

dnnmg_status dnnmg_net_create(const dnnmg_net_desc* net, const double* const* W, const double* const* scale,
                              const double* const* shift, int32_t precision, int64_t max_rows, void* cuda_stream,
                              dnnmg_ctx** out) {
    if (!out) return DNNMG_EINVAL;
    *out = nullptr;
    if (precision < DNNMG_FP64 || precision > DNNMG_BF16 || max_rows <= 0) return DNNMG_EINVAL;
    dnnmg_ctx* ctx = new (std::nothrow) dnnmg_ctx();
    if (!ctx) return DNNMG_ENOMEM;
    ctx->net_only = true;
    ctx->net_capacity = max_rows;
    // the input / output widths from the network: 216 or 1000 node values
    // (J = 1, 2) + 12 or 24 geometry features, 81 or 375 outputs
    if (net && net->widths && net->n_layers >= 1) {
        const bool j2 = net->widths[net->n_layers] == kNOutJ2;
        ctx->host.J = j2 ? 2 : 1;
        ctx->host.npn = j2 ? 125 : 27;
        ctx->host.n_geo = net->widths[0] - 8 * ctx->host.npn == 24 ? 24 : 12;
    }
    ctx->precision = precision;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        delete ctx;
        return DNNMG_ECUDA;
    }
    dnnmg_status st = dnnmg_set_network(ctx, net, W, scale, shift);
    if (st != DNNMG_OK) {
        dnnmg_destroy(ctx);
        return st;
    }
    *out = ctx;
    return DNNMG_OK;
}

dnnmg_status dnnmg_plain_step(dnnmg_ctx* ctx, int32_t level, int32_t n_steps, const dnnmg_solver_params* prm,
                              double* x_dev, dnnmg_solve_stats* stats) {
    Range nvtx_range("dnnmg_plain_step");
    if (!ctx || ctx->net_only || !x_dev || n_steps < 0) return DNNMG_EINVAL;
    DeviceLevel* L;
    dnnmg_status st = get_level(ctx, level, prm, &L);
    if (st != DNNMG_OK) return st;
    if (!ctx->plain_b[level] && (st = alloc(ctx, size_t(level_nodes(L)) * 4 * 8, &ctx->plain_b[level])) != DNNMG_OK)
        return st;
    void* b = ctx->plain_b[level];
    for (int32_t k = 0; k < n_steps; ++k) {
        if ((st = dnnmg_level_rhs(ctx, level, x_dev, (double*)b)) != DNNMG_OK) return st;
        st = dnnmg_solve(ctx, level, prm, (const double*)b, x_dev, stats);
        if (st != DNNMG_OK && st != DNNMG_ENOCONV) return st;
    }
    return DNNMG_OK;
}

}  // extern "C"
