// api.cu -- the C ABI (include/pdf_canyon.h): context life cycle, host-side
// mesh preprocessing, device memory, and the order of the kernel launches of
// one time step.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "pdf_internal.cuh"

static thread_local std::string g_init_error = "no error";

int fail(pdf_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return code;
}

void timing_begin(pdf_ctx* c, int k, cudaStream_t st) {
    if (!c->timing) return;
    std::pair<cudaEvent_t, cudaEvent_t> ev;
    if (!c->tm.pool.empty()) {
        ev = c->tm.pool.back();
        c->tm.pool.pop_back();
    } else {
        cudaEventCreate(&ev.first);
        cudaEventCreate(&ev.second);
    }
    cudaEventRecord(ev.first, st ? st : c->s);
    c->tm.ev[k].push_back(ev);
}

void timing_end(pdf_ctx* c, int k, cudaStream_t st) {
    if (!c->timing || c->tm.ev[k].empty()) return;
    cudaEventRecord(c->tm.ev[k].back().second, st ? st : c->s);
}

static void timing_collect(pdf_ctx* c) {
    for (int k = 0; k < PDF_K_COUNT; ++k) {
        for (auto& ev : c->tm.ev[k]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
                c->tm.total_ms[k] += ms;
                c->tm.launches[k] += 1;
            }
            c->tm.pool.push_back(ev);
        }
        c->tm.ev[k].clear();
    }
}

namespace {

template <typename T>
__global__ void k_to_double(const T* __restrict__ s, double* d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = (double)s[i];
}

template <typename T>
__global__ void k_from_double(const double* __restrict__ s, T* d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = (T)s[i];
}

__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

double orient(double px, double py, double qx, double qy, double rx, double ry) {
    return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

template <typename T>
int dalloc(pdf_ctx* c, T** p, size_t n) {
    if (n == 0) n = 1;
    PDF_CUDA(c, cudaMalloc((void**)p, sizeof(T) * n));
    return PDF_OK;
}

template <typename T>
int upload(pdf_ctx* c, T** p, const std::vector<T>& h) {
    int st = dalloc(c, p, h.size());
    if (st) return st;
    if (!h.empty()) PDF_CUDA(c, cudaMemcpy(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return PDF_OK;
}

#define TRY(x)                 \
    do {                       \
        int st_ = (x);         \
        if (st_ != PDF_OK) return st_; \
    } while (0)

int check_params(const pdf_params* p) {
    if (p->nb1 < 1 || p->nb2 < 1 || p->nb3 < 1 || p->nb1 * p->nb2 * p->nb3 > 255) return PDF_ERR_ARG;
    if (p->precision < 0 || p->precision > 2) return PDF_ERR_ARG;
    if (p->wall_model < 0 || p->wall_model > 1) return PDF_ERR_ARG;
    if (p->cg_precision < 0 || p->cg_precision > 1) return PDF_ERR_ARG;
    if (p->omega_wall < 0 || p->omega_wall > 1) return PDF_ERR_ARG;
    if (p->pressure < 0 || p->pressure > 1) return PDF_ERR_ARG;
    if (p->pressure && !(p->pressure_tol > 0.0 && p->pressure_tol < 1.0)) return PDF_ERR_ARG;
    if (!(p->period > 0) || !(p->nu > 0) || p->reflect_max < 0 || p->cg_maxit < 0) return PDF_ERR_ARG;
    return PDF_OK;
}

// host preprocessing of the mesh and upload
int build_mesh(pdf_ctx* c, const double* xy, int nn, const int* tri, int nt, const int* tag, const int* pair) {
    const double L = c->p.period;
    for (int i = 0; i < 3 * nt; ++i)
        if (tri[i] < 0 || tri[i] >= nn || tag[i] < 0 || tag[i] > 3) return fail(c, PDF_ERR_MESH, "node id or edge tag out of range");
    std::vector<int> rep(nn);
    for (int i = 0; i < nn; ++i) {
        const int q = pair[i];
        if (q >= nn || q == i || (q >= 0 && pair[q] != i)) return fail(c, PDF_ERR_MESH, "periodic pairs are not symmetric");
        if (q >= 0 && xy[2 * i + 1] != xy[2 * q + 1]) return fail(c, PDF_ERR_MESH, "periodic partners differ in y");
        rep[i] = (q >= 0 && q < i) ? q : i;
    }
    std::vector<double> area(nt), cent(2 * nt), gradb(6 * nt), egeo_d((size_t)EGEO_W * nt);
    std::vector<float> egeo_f((size_t)EGEO_W * nt);
    for (int e = 0; e < nt; ++e) {
        const int v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        const double A2 = orient(xy[2 * v[0]], xy[2 * v[0] + 1], xy[2 * v[1]], xy[2 * v[1] + 1], xy[2 * v[2]],
                                 xy[2 * v[2] + 1]);
        if (!(A2 > 0)) return fail(c, PDF_ERR_MESH, "triangle " + std::to_string(e) + " is not counter-clockwise");
        area[e] = 0.5 * A2;
        cent[2 * e] = (xy[2 * v[0]] + xy[2 * v[1]] + xy[2 * v[2]]) / 3.0;
        cent[2 * e + 1] = (xy[2 * v[0] + 1] + xy[2 * v[1] + 1] + xy[2 * v[2] + 1]) / 3.0;
        const double xr = xy[2 * v[0]], yr = xy[2 * v[0] + 1];
        const float xrf = (float)xr, yrf = (float)yr;
        egeo_d[EGEO_W * e] = xr; egeo_d[EGEO_W * e + 1] = yr;
        egeo_f[EGEO_W * e] = xrf; egeo_f[EGEO_W * e + 1] = yrf;
        for (int k = 0; k < 3; ++k) {
            const int a = v[(k + 1) % 3], b = v[(k + 2) % 3];
            const double ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1];
            const double gx = -(by - ay) / A2, gy = (bx - ax) / A2;
            gradb[6 * e + 2 * k] = gx;
            gradb[6 * e + 2 * k + 1] = gy;
            egeo_d[EGEO_W * e + 2 + 3 * k] = gx;
            egeo_d[EGEO_W * e + 3 + 3 * k] = gy;
            egeo_d[EGEO_W * e + 4 + 3 * k] = orient(ax, ay, bx, by, xr, yr) / A2;
            egeo_f[EGEO_W * e + 2 + 3 * k] = (float)gx;
            egeo_f[EGEO_W * e + 3 + 3 * k] = (float)gy;
            egeo_f[EGEO_W * e + 4 + 3 * k] = (float)(orient(ax, ay, bx, by, (double)xrf, (double)yrf) / A2);
        }
        egeo_d[EGEO_W * e + 11] = area[e];
        egeo_f[EGEO_W * e + 11] = (float)area[e];
    }
    // edge matching: interior edges by node pair, periodic edges by merged node pair
    struct Ed { long long k0, k1; int e, k; };
    std::vector<Ed> eds;
    eds.reserve(3 * (size_t)nt);
    for (int e = 0; e < nt; ++e)
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * e + (k + 1) % 3], b = tri[3 * e + (k + 2) % 3];
            if (tag[3 * e + k] == 3) { a = rep[a]; b = rep[b]; }
            eds.push_back({std::min(a, b), std::max(a, b), e, k});
        }
    std::sort(eds.begin(), eds.end(), [](const Ed& x, const Ed& y) {
        if (x.k0 != y.k0) return x.k0 < y.k0;
        if (x.k1 != y.k1) return x.k1 < y.k1;
        return x.e < y.e;
    });
    std::vector<int> nbr(3 * (size_t)nt, -1), einfo(nt, 0);
    for (size_t q = 0; q < eds.size();) {
        size_t r = q;
        while (r < eds.size() && eds[r].k0 == eds[q].k0 && eds[r].k1 == eds[q].k1) ++r;
        const int cntg = (int)(r - q);
        const int t0 = tag[3 * eds[q].e + eds[q].k];
        if (t0 == 0 || t0 == 3) {
            if (cntg != 2 || tag[3 * eds[q + 1].e + eds[q + 1].k] != t0)
                return fail(c, PDF_ERR_MESH, "interior/periodic edge without exactly one partner");
            for (int s = 0; s < 2; ++s) {
                const Ed& me = eds[q + s];
                const Ed& ot = eds[q + 1 - s];
                nbr[3 * me.e + me.k] = ot.e;
                int info = einfo[me.e];
                info |= (t0 & 3) << (2 * me.k);
                info |= (ot.k & 3) << (12 + 2 * me.k);
                if (t0 == 3) {
                    const int a = tri[3 * me.e + (me.k + 1) % 3];
                    const int code = xy[2 * a] < 0.5 * L ? 1 : 2;
                    info |= code << (6 + 2 * me.k);
                }
                einfo[me.e] = info;
            }
        } else {
            for (size_t s = q; s < r; ++s) einfo[eds[s].e] |= (t0 & 3) << (2 * eds[s].k);
            if (cntg != 1) return fail(c, PDF_ERR_MESH, "boundary edge shared by two elements");
        }
        q = r;
    }
    // node -> incident elements, periodic partners merged (increasing element id)
    std::vector<int> n2e_off(nn + 1, 0), n2e;
    for (int e = 0; e < nt; ++e)
        for (int k = 0; k < 3; ++k) {
            const int a = tri[3 * e + k];
            n2e_off[a + 1]++;
            if (pair[a] >= 0) n2e_off[pair[a] + 1]++;
        }
    for (int i = 0; i < nn; ++i) n2e_off[i + 1] += n2e_off[i];
    n2e.resize(n2e_off[nn]);
    {
        std::vector<int> fill(n2e_off.begin(), n2e_off.end() - 1);
        for (int e = 0; e < nt; ++e)
            for (int k = 0; k < 3; ++k) {
                const int a = tri[3 * e + k];
                n2e[fill[a]++] = e;
                if (pair[a] >= 0) n2e[fill[pair[a]]++] = e;
            }
    }
    // wall normals (class sums), wall nodes, wall distance
    std::vector<double> wn(2 * nn, 0.0), wdist(nn, 0.0);
    std::vector<unsigned char> is_wall(nn, 0);
    std::vector<std::array<double, 4>> wsegs;
    for (int e = 0; e < nt; ++e)
        for (int k = 0; k < 3; ++k) {
            if (tag[3 * e + k] != 1) continue;
            const int a = tri[3 * e + (k + 1) % 3], b = tri[3 * e + (k + 2) % 3];
            const double ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1];
            const double len = std::hypot(bx - ax, by - ay);
            const double nx = -(by - ay) / len, ny = (bx - ax) / len;
            for (int v : {a, b}) {
                const int r = rep[v];
                wn[2 * r] += nx; wn[2 * r + 1] += ny; is_wall[r] = 1;
            }
            wsegs.push_back({ax, ay, bx, by});
        }
    for (int i = 0; i < nn; ++i)
        if (rep[i] == i) {
            const double l = std::hypot(wn[2 * i], wn[2 * i + 1]);
            if (l > 0) { wn[2 * i] /= l; wn[2 * i + 1] /= l; }
        }
    for (int i = 0; i < nn; ++i) {
        const int r = rep[i];
        wn[2 * i] = wn[2 * r]; wn[2 * i + 1] = wn[2 * r + 1]; is_wall[i] = is_wall[r];
        const double px = xy[2 * i], py = xy[2 * i + 1];
        double best = INFINITY;
        for (const auto& sg : wsegs)
            for (int im = -1; im <= 1; ++im) {
                const double ax = sg[0] + im * L, ay = sg[1], bx = sg[2] + im * L, by = sg[3];
                const double dx = bx - ax, dy = by - ay;
                double t = ((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy);
                t = t < 0 ? 0 : (t > 1 ? 1 : t);
                const double d = std::hypot(px - (ax + t * dx), py - (ay + t * dy));
                best = d < best ? d : best;
            }
        wdist[i] = (std::isfinite(best) ? best : 0.0) + c->p.wall_offset;
    }
    DevMesh& m = c->m;
    m.nn = nn;
    m.nt = nt;
    TRY(upload(c, &m.tri, std::vector<int>(tri, tri + 3 * (size_t)nt)));
    TRY(upload(c, &m.nbr, nbr));
    TRY(upload(c, &m.einfo, einfo));
    TRY(upload(c, &m.xy, std::vector<double>(xy, xy + 2 * (size_t)nn)));
    TRY(upload(c, &m.egeo_d, egeo_d));
    TRY(upload(c, &m.egeo_f, egeo_f));
    TRY(upload(c, &m.gradb, gradb));
    TRY(upload(c, &m.area, area));
    TRY(upload(c, &m.cent, cent));
    TRY(upload(c, &m.n2e_off, n2e_off));
    TRY(upload(c, &m.n2e, n2e));
    TRY(upload(c, &m.wdist, wdist));
    TRY(upload(c, &m.wn, wn));
    TRY(upload(c, &m.is_wall, is_wall));
    TRY(upload(c, &m.rep, rep));
    // Section 4 frequency reflection: wall nodes and the elements around them
    if (c->p.wall_model == PDF_WALL_FUNCTIONS && c->p.omega_wall) {
        std::vector<int> wnodes, welems;
        std::vector<unsigned char> mark(nt, 0);
        for (int i = 0; i < nn; ++i) {
            if (!is_wall[i]) continue;
            wnodes.push_back(i);
            for (int q = n2e_off[i]; q < n2e_off[i + 1]; ++q) mark[n2e[q]] = 1;
        }
        for (int e = 0; e < nt; ++e)
            if (mark[e]) welems.push_back(e);
        m.n_owall_node = (int)wnodes.size();
        m.n_owall_elem = (int)welems.size();
        TRY(upload(c, &m.owall_node, wnodes));
        TRY(upload(c, &m.owall_elem, welems));
    }
    // finite-element pattern over canonical nodes (elliptic relaxation and
    // the pressure projection)
    if (c->p.wall_model == PDF_ELLIPTIC_RELAXATION || c->p.pressure) {
        std::vector<std::pair<long long, int>> ent;  // (row*nn + col, contribution id)
        ent.reserve(9 * (size_t)nt);
        std::vector<double> mloc(9 * (size_t)nt), kloc(9 * (size_t)nt);
        std::vector<int> celem(9 * (size_t)nt);
        for (int e = 0; e < nt; ++e)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    const int id = 9 * e + 3 * k + l;
                    const long long r = rep[tri[3 * e + k]], col = rep[tri[3 * e + l]];
                    ent.push_back({r * nn + col, id});
                    mloc[id] = area[e] / 12.0 * (k == l ? 2.0 : 1.0);
                    kloc[id] = area[e] * (gradb[6 * e + 2 * k] * gradb[6 * e + 2 * l] +
                                          gradb[6 * e + 2 * k + 1] * gradb[6 * e + 2 * l + 1]);
                    celem[id] = e;
                }
        std::sort(ent.begin(), ent.end());
        std::vector<int> rowptr(nn + 1, 0), colidx, kc_off(1, 0), kc_elem, diag(nn, -1);
        std::vector<double> mval, kc_geo;
        for (size_t q = 0; q < ent.size();) {
            size_t r = q;
            double ms = 0.0;
            while (r < ent.size() && ent[r].first == ent[q].first) {
                ms += mloc[ent[r].second];
                kc_elem.push_back(celem[ent[r].second]);
                kc_geo.push_back(kloc[ent[r].second]);
                ++r;
            }
            const int row = (int)(ent[q].first / nn), col = (int)(ent[q].first % nn);
            if (row == col) diag[row] = (int)colidx.size();
            colidx.push_back(col);
            mval.push_back(ms);
            kc_off.push_back((int)kc_elem.size());
            rowptr[row + 1]++;
            q = r;
        }
        for (int i = 0; i < nn; ++i) rowptr[i + 1] += rowptr[i];
        m.nnz = (int)colidx.size();
        TRY(upload(c, &m.rowptr, rowptr));
        TRY(upload(c, &m.colidx, colidx));
        TRY(upload(c, &m.mval, mval));
        TRY(upload(c, &m.kc_off, kc_off));
        TRY(upload(c, &m.kc_elem, kc_elem));
        TRY(upload(c, &m.kc_geo, kc_geo));
        TRY(upload(c, &m.diag, diag));
        TRY(dalloc(c, &m.aval, m.nnz));
        TRY(dalloc(c, &m.avf, m.nnz));
        if (c->p.pressure) {
            // stiffness sum_e A_e grad N_k . grad N_l, and p = 0 at the lowest-id canonical node
            std::vector<double> pval(m.nnz, 0.0);
            for (int q = 0; q < m.nnz; ++q)
                for (int r = kc_off[q]; r < kc_off[q + 1]; ++r) pval[q] += kc_geo[r];
            std::vector<unsigned char> pin(nn, 0);
            for (int i = 0; i < nn; ++i)
                if (rep[i] == i) { pin[i] = 1; break; }
            TRY(upload(c, &m.pval, pval));
            TRY(upload(c, &m.pin, pin));
        }
    }
    return PDF_OK;
}

int alloc_stats(pdf_ctx* c) {
    const int nn = c->m.nn, nt = c->m.nt, B = c->B;
    const size_t ts = c->prec == 0 ? 8 : 4;
    TRY(dalloc(c, &c->cnt, nt));
    TRY(dalloc(c, &c->off, nt + 1));
    TRY(dalloc(c, &c->cursor, nt));
    TRY(dalloc(c, &c->scan_part, scan_blocks(nt) + 1));
    TRY(dalloc(c, &c->en, nt));
    TRY(dalloc(c, &c->emean, 5 * (size_t)nt));
    TRY(dalloc(c, &c->eR, 6 * (size_t)nt));
    TRY(dalloc(c, &c->epsivar, nt));
    TRY(dalloc(c, &c->ecm, (size_t)B * nt));
    TRY(dalloc(c, &c->elist, 8 + 2 * (size_t)nt));  // 8 counters, then the two lists
    TRY(dalloc(c, &c->nwt, nn));
    TRY(dalloc(c, &c->nmean, 4 * (size_t)nn));
    TRY(dalloc(c, &c->nR, 6 * (size_t)nn));
    TRY(dalloc(c, &c->nke, 2 * (size_t)nn));
    TRY(dalloc(c, &c->npsivar, nn));
    TRY(dalloc(c, &c->eder, 9 * (size_t)nt));
    TRY(dalloc(c, &c->ngrad, 4 * (size_t)nn));
    TRY(dalloc(c, &c->npack, 11 * (size_t)nn));
    TRY(dalloc(c, &c->nwp, 5 * (size_t)nn));
    if (c->m.n_owall_elem > 0) {
        TRY(dalloc(c, &c->eomw, 5 * (size_t)nt));
        TRY(dalloc(c, &c->nomw, 5 * (size_t)nn));
        PDF_CUDA(c, cudaMemset(c->eomw, 0, sizeof(double) * 5 * nt));
        PDF_CUDA(c, cudaMemset(c->nomw, 0, sizeof(double) * 5 * nn));
    }
    PDF_CUDA(c, cudaMalloc(&c->npackT, ts * NODE_PACK_W * nn));
    PDF_CUDA(c, cudaMalloc(&c->epackT, ts * ELEM_PACK_W * nt));
    PDF_CUDA(c, cudaMalloc(&c->eaffT, ts * ELEM_AFF_W * nt));
    PDF_CUDA(c, cudaMalloc(&c->ecmT, ts * (size_t)B * nt));
    // node statistics start at zero (a node without particles keeps its old value)
    PDF_CUDA(c, cudaMemset(c->nmean, 0, sizeof(double) * 4 * nn));
    PDF_CUDA(c, cudaMemset(c->nR, 0, sizeof(double) * 6 * nn));
    PDF_CUDA(c, cudaMemset(c->nke, 0, sizeof(double) * 2 * nn));
    PDF_CUDA(c, cudaMemset(c->npsivar, 0, sizeof(double) * nn));
    PDF_CUDA(c, cudaMemset(c->nwp, 0, sizeof(double) * 5 * nn));
    TRY(dalloc(c, &c->d_status, 1));
    TRY(dalloc(c, &c->d_step, 1));
    PDF_CUDA(c, cudaMemset(c->d_step, 0, sizeof(uint32_t)));
    PDF_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
    PDF_CUDA(c, cudaMallocHost((void**)&c->h_status, sizeof(int)));
    if (c->p.wall_model == PDF_ELLIPTIC_RELAXATION || c->p.pressure) {
        const size_t v = 5 * (size_t)nn;
        if (c->p.wall_model == PDF_ELLIPTIC_RELAXATION) {
            TRY(dalloc(c, &c->fe_f, v));
            TRY(dalloc(c, &c->fe_g, v));
            TRY(dalloc(c, &c->fe_prop, v));
            PDF_CUDA(c, cudaMemset(c->fe_g, 0, sizeof(double) * v));
        }
        if (c->p.pressure) {
            TRY(dalloc(c, &c->pr_b, nn));
            TRY(dalloc(c, &c->pr_x, nn));
            TRY(dalloc(c, &c->pres, nn));
            TRY(dalloc(c, &c->egp, 2 * (size_t)nt));
            TRY(dalloc(c, &c->pr_iters, 1));
            PDF_CUDA(c, cudaMemset(c->pr_b, 0, sizeof(double) * nn));
            PDF_CUDA(c, cudaMemset(c->pr_x, 0, sizeof(double) * nn));
            PDF_CUDA(c, cudaMemset(c->pres, 0, sizeof(double) * nn));
            PDF_CUDA(c, cudaMemset(c->pr_iters, 0, sizeof(int)));
        }
        TRY(dalloc(c, &c->fe_z, v));
        TRY(dalloc(c, &c->fe_part, (size_t)15 * 4096));
        TRY(dalloc(c, &c->fe_bar, 32 * 64));  // barrier lines: top/generation + 63 groups of 16 blocks
        PDF_CUDA(c, cudaMemset(c->fe_bar, 0, 32 * 64 * sizeof(unsigned)));
        TRY(dalloc(c, &c->fe_iters, 1));
        PDF_CUDA(c, cudaMemset(c->fe_iters, 0, sizeof(int)));
    }
    return PDF_OK;
}

int alloc_particles(pdf_ctx* c, int64_t n) {
    if (n <= c->cap) {
        c->np = n;
        return PDF_OK;
    }
    for (int k = 0; k < 7; ++k) {
        cudaFree(c->stA[k]);
        cudaFree(c->stB[k]);
        c->stA[k] = c->stB[k] = nullptr;
    }
    cudaFree(c->idA); cudaFree(c->idB); cudaFree(c->elemA); cudaFree(c->elemB); cudaFree(c->bin);
    cudaFree(c->sort_scratch); cudaFree(c->conv_buf);
    c->idA = c->idB = nullptr;
    c->elemA = c->elemB = nullptr;
    c->bin = nullptr;
    c->sort_scratch = nullptr;
    c->conv_buf = nullptr;
    c->cap = 0;
    const size_t ts = c->prec == 0 ? 8 : 4;
    // whole tiles of 256 particles: the particle kernel stages tiles with
    // 16-byte-granular bulk copies that may run past n inside the allocation
    const int64_t na = (n + 255) / 256 * 256;
    for (int k = 0; k < 7; ++k) {
        PDF_CUDA(c, cudaMalloc(&c->stA[k], ts * na));
        PDF_CUDA(c, cudaMalloc(&c->stB[k], ts * na));
    }
    TRY(dalloc(c, &c->idA, na));
    TRY(dalloc(c, &c->idB, na));
    TRY(dalloc(c, &c->elemA, na));
    TRY(dalloc(c, &c->elemB, na));
    TRY(dalloc(c, &c->bin, na));
    PDF_CUDA(c, cudaMemset(c->bin, 0, na));
    TRY(dalloc(c, &c->sort_scratch, 2 * (size_t)n));
    c->sort_scratch_n = 2 * n;
    c->conv_bytes = sizeof(double) * (size_t)n;
    PDF_CUDA(c, cudaMalloc(&c->conv_buf, c->conv_bytes));
    c->cap = n;
    c->np = n;
    return PDF_OK;
}

}  // namespace

int set_device_step(pdf_ctx* c) {
    k_set_u32<<<1, 1, 0, c->s>>>(c->d_step, (uint32_t)c->step);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

int launch_to_double(pdf_ctx* c, const void* src, double* dst, int64_t n) {
    if (n == 0) return PDF_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (c->prec == 0) k_to_double<double><<<blocks, 256, 0, c->s>>>((const double*)src, dst, n);
    else k_to_double<float><<<blocks, 256, 0, c->s>>>((const float*)src, dst, n);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

extern "C" {

int pdf_default_params(pdf_params* p) {
    if (!p) return PDF_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    // Table 2
    p->C1 = 1.85; p->C2 = 0.63; p->C3 = 5.0; p->C4 = 0.25; p->CT = 6.0; p->CL = 0.134; p->Ceta = 72.0;
    p->Cv = 1.4; p->gamma5 = 0.1; p->Comega1 = 0.5; p->Comega2 = 0.73; p->Cs = 0.02; p->Ct = 0.7;
    // Section 2.2
    p->C0 = 3.5; p->Cmu = 0.09; p->kappa = 0.41; p->E = 8.5;
    // Section 3 set-up: Re = 12000 on U0 = H = 1, u* = 0.05 drives the flow
    p->nu = 1.0 / 12000.0;
    p->ustar = 0.05;
    p->fx = p->ustar * p->ustar / 1.0;
    p->fy = 0.0;
    p->yp = 30.0 * p->nu / p->ustar;
    p->wall_offset = 0.0;
    p->x0 = 1.5; p->y0 = 0.0; p->r0 = 0.05;
    p->period = 3.0;
    p->k0 = 1e-3; p->y_roof = 1.0;
    p->er_wall = 4.5;
    p->floor_k = 1e-12; p->floor_eps = 1e-12; p->floor_omega = 1e-12;
    p->cg_tol = 1e-8; p->cg_maxit = 2000;
    p->nb1 = 2; p->nb2 = 2; p->nb3 = 2;
    p->wall_model = PDF_WALL_FUNCTIONS;
    p->mix_exp = 0;
    p->reflect_max = 8;
    p->rotta = 0;
    p->seed = 0;
    p->case_id = 0;
    p->precision = PDF_FP64;
    p->cg_precision = 0;
    p->omega_wall = 0;
    p->pressure = 0;
    p->reserved_ = 0;
    p->pressure_tol = 1e-6;
    return PDF_OK;
}

int pdf_init_mesh(const pdf_params* p, const double* xy, int32_t nnode, const int32_t* tri, int32_t ntri,
                  const int32_t* edge_tag, const int32_t* periodic_pair, void* cuda_stream, pdf_ctx** out) {
    if (!out) return fail(nullptr, PDF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !xy || !tri || !edge_tag || !periodic_pair || nnode < 3 || ntri < 1)
        return fail(nullptr, PDF_ERR_ARG, "NULL pointer or empty mesh");
    if (check_params(p) != PDF_OK) return fail(nullptr, PDF_ERR_ARG, "invalid parameters");
    pdf_ctx* c = new pdf_ctx();
    c->p = *p;
    c->B = p->nb1 * p->nb2 * p->nb3;
    c->prec = p->precision;
    c->s = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int st = build_mesh(c, xy, nnode, tri, ntri, edge_tag, periodic_pair);
    if (st == PDF_OK) st = alloc_stats(c);
    if (st == PDF_OK) st = prepare_moments(c);
    if (st == PDF_OK && c->p.pressure) st = prepare_pressure(c);
    if (st != PDF_OK) {
        g_init_error = c->err;
        pdf_destroy(c);
        return st;
    }
    *out = c;
    return PDF_OK;
}

int pdf_seed_particles(pdf_ctx* c, int32_t per_element) {
    if (!c || per_element < 0) return PDF_ERR_ARG;
    const int64_t n = (int64_t)c->m.nt * per_element;
    if (n > 0xffffffffll) return fail(c, PDF_ERR_CAPACITY, "more than 2^32 particles");
    TRY(alloc_particles(c, n));
    TRY(launch_seed(c, per_element));
    TRY(launch_count_and_sort(c));
    c->step = 0;
    TRY(set_device_step(c));
    c->seeded = true;
    c->stats_valid = false;
    return PDF_OK;
}

int pdf_set_particles(pdf_ctx* c, int32_t n, const double* x, const double* y, const double* u, const double* v,
                      const double* w, const double* omega, const double* psi, const uint32_t* id,
                      const int32_t* elem, int32_t step) {
    if (!c || n < 0 || (n > 0 && (!x || !y || !u || !v || !w || !omega || !psi || !id || !elem)) || step < 0)
        return c ? fail(c, PDF_ERR_ARG, "bad particle arrays") : PDF_ERR_ARG;
    TRY(alloc_particles(c, n));
    const double* src[7] = {x, y, u, v, w, omega, psi};
    const unsigned blocks = (unsigned)((n + 255) / 256);
    for (int k = 0; k < 7 && n > 0; ++k) {
        PDF_CUDA(c, cudaMemcpyAsync(c->conv_buf, src[k], sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
        if (c->prec == 0)
            PDF_CUDA(c, cudaMemcpyAsync(c->stA[k], c->conv_buf, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
        else
        {
            k_from_double<float><<<blocks, 256, 0, c->s>>>((const double*)c->conv_buf, (float*)c->stA[k], n);
            ++c->launches;
        }
    }
    if (n > 0) {
        PDF_CUDA(c, cudaMemcpyAsync(c->idA, id, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, c->s));
        PDF_CUDA(c, cudaMemcpyAsync(c->elemA, elem, sizeof(int) * n, cudaMemcpyHostToDevice, c->s));
    }
    TRY(launch_count_and_sort(c));
    const int st = pdf_sync(c);
    if (st == PDF_ERR_CAPACITY) return fail(c, PDF_ERR_ARG, "element id out of range");
    if (st != PDF_OK) return st;
    c->step = step;
    TRY(set_device_step(c));
    c->seeded = true;
    c->stats_valid = false;
    return PDF_OK;
}

int pdf_estimate_stats(pdf_ctx* c) {
    if (!c) return PDF_ERR_ARG;
    if (!c->seeded) return fail(c, PDF_ERR_STATE, "no particles");
    TRY(launch_moments(c));
    TRY(launch_fields(c));
    TRY(join_bins(c));
    c->stats_valid = true;
    return PDF_OK;
}

int pdf_step(pdf_ctx* c, double dt, int32_t nsteps) {
    if (!c) return PDF_ERR_ARG;
    if (!(dt > 0) || nsteps < 0) return fail(c, PDF_ERR_ARG, "dt must be positive and nsteps >= 0");
    if (!c->stats_valid) return fail(c, PDF_ERR_STATE, "statistics not estimated");
    for (int s = 0; s < nsteps; ++s) {
        TRY(launch_particle_step(c, dt));
        TRY(launch_sort(c, true));
        c->step++;
        TRY(launch_moments(c));
        if (c->p.pressure) {  // the projection moves the velocities the bins read
            TRY(join_bins(c));
            TRY(launch_pressure(c, dt));
        }
        TRY(launch_fields(c));
        TRY(join_bins(c));
        TRY(launch_averaging(c));
    }
    return PDF_OK;
}

int pdf_set_wait_limit(pdf_ctx* c, int64_t spins) {
    if (!c || spins < 0) return PDF_ERR_ARG;
    c->wait_spins = (long long)spins;
    return PDF_OK;
}

int pdf_sync(pdf_ctx* c) {
    if (!c) return PDF_ERR_ARG;
    TRY(join_bins(c));  // (left pending only by a launch that failed)
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    PDF_CUDA(c, cudaMemcpy(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    const int s = *c->h_status;
    if (s) PDF_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (s & ST_BARRIER) {
        // a block that gave up left the barrier's arrival count behind: the
        // stream is idle, so start the solver's barrier words afresh
        if (c->fe_bar) PDF_CUDA(c, cudaMemset(c->fe_bar, 0, 32 * 64 * sizeof(unsigned)));
        return fail(c, PDF_ERR_CUDA, "grid barrier of the elliptic solver timed out");
    }
    if (s & ST_NONFINITE) return fail(c, PDF_ERR_NONFINITE, "non-finite particle state");
    if (s & ST_LOST) return fail(c, PDF_ERR_LOST_PARTICLE, "element walk exceeded its cap");
    if (s & ST_WALL) return fail(c, PDF_ERR_WALL, "too many boundary reflections in one step");
    if (s & ST_DT) return fail(c, PDF_ERR_DT, "Euler mixing ratio dt/t_m above one");
    if (s & ST_CG) return fail(c, PDF_ERR_CG_NOCONV, "elliptic-relaxation CG did not converge");
    if (s & ST_CAPACITY) return fail(c, PDF_ERR_CAPACITY, "capacity exceeded");
    return PDF_OK;
}

}  // extern "C"

// device source, size in bytes and FP64 conversion of a field (the mapping
// behind pdf_get_fields; also used to check a batch's output sizes)
int field_source(pdf_ctx* c, int32_t field, const void** src_out, size_t* need_out, bool* convert_out) {
    const int64_t n = c->np;
    const int nt = c->m.nt, nn = c->m.nn;
    const void* src = nullptr;
    size_t need = 0;
    bool convert = false;
    switch (field) {
    case PDF_FIELD_X: case PDF_FIELD_Y: case PDF_FIELD_U: case PDF_FIELD_V: case PDF_FIELD_W:
    case PDF_FIELD_OMEGA: case PDF_FIELD_PSI:
        src = c->stA[field - PDF_FIELD_X]; need = 8 * (size_t)n; convert = true; break;
    case PDF_FIELD_ID: src = c->idA; need = 4 * (size_t)n; break;
    case PDF_FIELD_ELEM: src = c->elemA; need = 4 * (size_t)n; break;
    case PDF_FIELD_BIN: src = c->bin; need = (size_t)n; break;
    case PDF_FIELD_ELEM_N: src = c->en; need = 4 * (size_t)nt; break;
    case PDF_FIELD_ELEM_MEAN: src = c->emean; need = 8 * 5 * (size_t)nt; break;
    case PDF_FIELD_ELEM_R: src = c->eR; need = 8 * 6 * (size_t)nt; break;
    case PDF_FIELD_ELEM_PSIVAR: src = c->epsivar; need = 8 * (size_t)nt; break;
    case PDF_FIELD_ELEM_CM: src = c->ecm; need = 8 * (size_t)c->B * nt; break;
    case PDF_FIELD_NODE_MEAN: src = c->nmean; need = 8 * 4 * (size_t)nn; break;
    case PDF_FIELD_NODE_R: src = c->nR; need = 8 * 6 * (size_t)nn; break;
    case PDF_FIELD_NODE_KE: src = c->nke; need = 8 * 2 * (size_t)nn; break;
    case PDF_FIELD_ELEM_DER: src = c->eder; need = 8 * 9 * (size_t)nt; break;
    case PDF_FIELD_NODE_PACK: src = c->npack; need = 8 * 11 * (size_t)nn; break;
    case PDF_FIELD_NODE_WP: src = c->nwp; need = 8 * 5 * (size_t)nn; break;
    case PDF_FIELD_NODE_WDIST: src = c->m.wdist; need = 8 * (size_t)nn; break;
    case PDF_FIELD_NODE_GRAD: src = c->ngrad; need = 8 * 4 * (size_t)nn; break;
    case PDF_FIELD_NODE_PSIVAR: src = c->npsivar; need = 8 * (size_t)nn; break;
    case PDF_FIELD_ELEM_OMW: case PDF_FIELD_NODE_OMW:
        if (!c->eomw) return fail(c, PDF_ERR_STATE, "frequency-weighted wall moments exist with omega_wall = 1 only");
        if (field == PDF_FIELD_ELEM_OMW) { src = c->eomw; need = 8 * 5 * (size_t)nt; }
        else { src = c->nomw; need = 8 * 5 * (size_t)nn; }
        break;
    case PDF_FIELD_NODE_P:
        if (!c->pres) return fail(c, PDF_ERR_STATE, "the projection pressure exists with pressure = 1 only");
        src = c->pres; need = 8 * (size_t)nn; break;
    case PDF_FIELD_PARTICLE_WP:
        if (c->sur_mode != 4 || !c->pwp || c->pwp_n < n)
            return fail(c, PDF_ERR_STATE, "particle wp is recorded in surrogate mode 4 only");
        src = c->pwp; need = 4 * 5 * (size_t)n; break;
    default: return fail(c, PDF_ERR_ARG, "unknown field id");
    }
    *src_out = src;
    *need_out = need;
    *convert_out = convert;
    return PDF_OK;
}

extern "C" {

int pdf_get_fields(pdf_ctx* c, int32_t field, void* dst, size_t bytes, int32_t dst_is_device) {
    if (!c || !dst || dst_is_device < 0 || dst_is_device > 2) return PDF_ERR_ARG;
    const int64_t n = c->np;
    const void* src = nullptr;
    size_t need = 0;
    bool convert = false;
    TRY(field_source(c, field, &src, &need, &convert));
    if (bytes != need) return fail(c, PDF_ERR_ARG, "field size mismatch: expected " + std::to_string(need));
    if (need == 0) return PDF_OK;
    if (convert) {
        if (c->prec == 0) {
            // already double
        } else {
            TRY(launch_to_double(c, src, (double*)c->conv_buf, n));
            src = c->conv_buf;
        }
    }
    PDF_CUDA(c, cudaMemcpyAsync(dst, src, need, dst_is_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->s));
    if (dst_is_device == 0) PDF_CUDA(c, cudaStreamSynchronize(c->s));
    return PDF_OK;
}

int64_t pdf_num_particles(const pdf_ctx* c) { return c ? c->np : -1; }
int32_t pdf_num_elements(const pdf_ctx* c) { return c ? c->m.nt : -1; }
int32_t pdf_num_nodes(const pdf_ctx* c) { return c ? c->m.nn : -1; }
int32_t pdf_num_bins(const pdf_ctx* c) { return c ? c->B : -1; }
int32_t pdf_step_index(const pdf_ctx* c) { return c ? c->step : -1; }

int32_t pdf_pressure_iterations(pdf_ctx* c) {
    if (!c || !c->pr_iters) return 0;
    int it = 0;
    if (cudaMemcpy(&it, c->pr_iters, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return it;
}

int32_t pdf_cg_iterations(pdf_ctx* c) {
    if (!c || !c->fe_iters) return 0;
    int it = 0;
    if (cudaMemcpy(&it, c->fe_iters, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return it;
}

int pdf_set_timing(pdf_ctx* c, int32_t on) {
    if (!c) return PDF_ERR_ARG;
    c->timing = on ? 1 : 0;
    return PDF_OK;
}

int pdf_kernel_time(pdf_ctx* c, int32_t kernel, double* total_ms, int64_t* launches) {
    if (!c || kernel < 0 || kernel >= PDF_K_COUNT || !total_ms || !launches) return PDF_ERR_ARG;
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    timing_collect(c);
    *total_ms = c->tm.total_ms[kernel];
    *launches = c->tm.launches[kernel];
    return PDF_OK;
}

int pdf_reset_timing(pdf_ctx* c) {
    if (!c) return PDF_ERR_ARG;
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    timing_collect(c);
    for (int k = 0; k < PDF_K_COUNT; ++k) {
        c->tm.total_ms[k] = 0;
        c->tm.launches[k] = 0;
    }
    return PDF_OK;
}

int64_t pdf_launch_count(const pdf_ctx* c) { return c ? c->launches : -1; }

const char* pdf_last_error(const pdf_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

void pdf_destroy(pdf_ctx* c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    else cudaDeviceSynchronize();
    timing_collect(c);
    for (auto& ev : c->tm.pool) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    DevMesh& m = c->m;
    void* dev[] = {m.tri, m.nbr, m.einfo, m.xy, m.egeo_d, m.egeo_f, m.gradb, m.area, m.cent, m.n2e_off, m.n2e,
                   m.wdist, m.wn, m.is_wall, m.rep, m.rowptr, m.colidx, m.mval, m.kc_off, m.kc_elem, m.kc_geo,
                   m.aval, m.avf, m.diag, m.owall_node, m.owall_elem, m.pval, m.pin, c->eomw, c->nomw, c->pr_b, c->pr_x, c->pr_binv,
                   c->pr_a0inv, c->pres, c->egp, c->pr_iters, c->idA, c->idB, c->elemA, c->elemB, c->bin, c->cnt, c->off, c->cursor, c->scan_part, c->en,
                   c->emean, c->eR, c->epsivar, c->ecm, c->nwt, c->nmean, c->nR, c->nke, c->npsivar, c->eder,
                   c->ngrad, c->npack, c->nwp, c->npackT, c->epackT, c->eaffT, c->ecmT, c->sort_scratch, c->fe_f, c->fe_g,
                   c->fe_prop, c->fe_z, c->fe_part, c->fe_bar, c->fe_iters, c->d_status,
                   c->conv_buf, c->elist, c->d_step, c->nsurT, c->pwp, c->avg_sum, c->avg_count, c->cdf_elem, c->cdf_hist, c->sur_w, c->sur_rows, c->sur_skip, c->sur_cnt, c->sur_part, c->sur_base, c->sur_snap, c->sur_y};
    for (void* p : dev) cudaFree(p);
    for (int k = 0; k < 7; ++k) {
        cudaFree(c->stA[k]);
        cudaFree(c->stB[k]);
    }
    cudaFreeHost(c->h_status);
    if (c->side_fork) cudaEventDestroy(c->side_fork);
    if (c->side_join) cudaEventDestroy(c->side_join);
    if (c->side_join2) cudaEventDestroy(c->side_join2);
    if (c->s2) cudaStreamDestroy(c->s2);
    if (c->bins_join) cudaEventDestroy(c->bins_join);
    if (c->crowd_done) cudaEventDestroy(c->crowd_done);
    if (c->s3) cudaStreamDestroy(c->s3);
    if (c->s_cond) cudaStreamDestroy(c->s_cond);
    delete c;
}

}  // extern "C"
