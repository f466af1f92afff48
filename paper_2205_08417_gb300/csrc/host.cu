// kitrt host side: mesh construction, angular tables, workspace, and the C ABI entry points.
//
// Mesh [Sec. 4.1]: cell-centred triangles with area, neighbours and length-scaled outward
// normals. Angular tables [Sec. 3.1, Sec. 3.2]: product quadrature (Gauss-Legendre in mu x
// uniform azimuth), real spherical harmonics even in mu, folded over +-mu. The Hessian of the
// dual is assembled from moments against the degree-2N basis through Gaunt coefficients
// <m_a m_b m~_c>, which is exact because a product of two harmonics of degree <= N is a
// combination of harmonics of degree <= 2N (and stays even in mu).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "kitrt_internal.cuh"

namespace {

const double kPi = 3.14159265358979323846;

#define CUDA_OK(x)                                   \
    do {                                             \
        if ((x) != cudaSuccess) return KITRT_ECUDA; \
    } while (0)

// Gauss-Legendre rule on [-1,1] (ascending nodes): Newton iteration on P_n(x), evaluated by the
// Bonnet recurrence, from Tricomi's initial approximation of the k-th root.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 1; k <= n; ++k) {
        double th = kPi * (4.0 * k - 1.0) / (4.0 * n + 2.0);
        double r = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
        double dpn = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm = 1.0, pc = r;
            for (int j = 2; j <= n; ++j) {
                double pn = ((2 * j - 1) * r * pc - (j - 1) * pm) / j;
                pm = pc;
                pc = pn;
            }
            if (n == 1) pm = 1.0, pc = r;
            dpn = n * (pm - r * pc) / (1.0 - r * r);
            double step = pc / dpn;
            r -= step;
            if (fabs(step) <= 1e-17) break;
        }
        double pm = 1.0, pc = r;
        for (int j = 2; j <= n; ++j) {
            double pn = ((2 * j - 1) * r * pc - (j - 1) * pm) / j;
            pm = pc;
            pc = pn;
        }
        dpn = n * (pm - r * pc) / (1.0 - r * r);
        // root k counted from +1 downwards
        x[n - k] = r;
        w[n - k] = 2.0 / ((1.0 - r * r) * dpn * dpn);
    }
}

// Fully normalised associated Legendre values Pn[l][k] = N_l^k P_l^k(mu) (no Condon-Shortley
// phase) for 0 <= k <= l <= L, by the standard stable recurrences in l.
void norm_legendre(int L, double mu, double Pn[][24])
{
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    Pn[0][0] = 1.0 / sqrt(4.0 * kPi);
    for (int k = 1; k <= L; ++k) Pn[k][k] = sqrt((2.0 * k + 1.0) / (2.0 * k)) * s * Pn[k - 1][k - 1];
    for (int k = 0; k < L; ++k) Pn[k + 1][k] = sqrt(2.0 * k + 3.0) * mu * Pn[k][k];
    for (int k = 0; k <= L; ++k)
        for (int l = k + 2; l <= L; ++l) {
            double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)k * k));
            double b = sqrt((((l - 1.0) * (l - 1.0)) - (double)k * k) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            Pn[l][k] = a * (mu * Pn[l - 1][k] - b * Pn[l - 2][k]);
        }
}

// 2D basis of degree L at (mu, phi): real harmonics m_l^k with l + |k| even, ordered by l then k.
int basis2d(int L, double mu, double phi, double *out)
{
    double Pn[24][24];
    norm_legendre(L, mu, Pn);
    int i = 0;
    for (int l = 0; l <= L; ++l)
        for (int k = -l; k <= l; ++k) {
            int ak = k < 0 ? -k : k;
            if ((l + ak) % 2) continue;
            double v = Pn[l][ak];
            if (k > 0) v *= sqrt(2.0) * cos(k * phi);
            if (k < 0) v *= sqrt(2.0) * sin(ak * phi);
            out[i++] = v;
        }
    return i;
}

int nmom_of(int L) { return (L + 1) * (L + 2) / 2; }

// Folded product rule: pairs of Gauss nodes +-mu share the 2D direction and every basis value,
// so they merge into one point of doubled weight (an odd order keeps mu = 0 once). Each ring (one
// |mu|) has nphi = 2 order equally spaced azimuths phi_l = l 2 pi / nphi, l = 1..nphi, stored as
// P = nphi / 2 pairs of points: pair 0 = (phi = 2 pi, phi = pi), the two azimuths whose sines
// vanish; pair j >= 1 = (phi_j, phi_{nphi-j} = 2 pi - phi_j), a direction and its mirror image,
// whose cosines are equal and whose sines are opposite. Pairs of a ring are consecutive, and
// the two points of a pair are consecutive.
struct FoldedRule {
    std::vector<double> mu, phi, w;  // per point
    std::vector<int> kind;           // per point: 0 first of a mirror pair, 1 its mirror,
                                     // 2 phi = 0 (= 2 pi), 3 phi = pi
    std::vector<double> ring_mu, ring_w;  // per ring: |mu| and the weight of each of its points
    int nphi = 0, P = 0;
};

FoldedRule folded_rule(int order)
{
    std::vector<double> x, gw;
    gauss_legendre(order, x, gw);
    const int nphi = 2 * order, half = order / 2;
    FoldedRule r;
    r.nphi = nphi;
    r.P = nphi / 2;
    auto add_ring = [&](double mu, double wk) {
        const double wpt = wk * 2.0 * kPi / nphi;
        r.ring_mu.push_back(mu);
        r.ring_w.push_back(wpt);
        auto add = [&](double phi, int kind) {
            r.mu.push_back(mu);
            r.phi.push_back(phi);
            r.w.push_back(wpt);
            r.kind.push_back(kind);
        };
        add(2.0 * kPi, 2);
        add(kPi, 3);
        for (int j = 1; j < nphi / 2; ++j) {
            add(j * (2.0 * kPi / nphi), 0);
            add((nphi - j) * (2.0 * kPi / nphi), 1);
        }
    };
    // nodes are ascending: k = order-1 .. order-half are the positive ones, paired with order-1-k
    for (int k = order - 1; k >= order - half; --k) add_ring(x[k], gw[k] + gw[order - 1 - k]);
    if (order % 2) add_ring(0.0, gw[half]);
    return r;
}

// Azimuthal factor T_k(phi) of the real harmonics: 1 (k = 0), sqrt2 cos(k phi) (k > 0),
// sqrt2 sin(|k| phi) (k < 0), with the symmetries of the pairs made exact: the mirror point takes
// the first point's values with the sines negated, and phi = 0 and phi = pi take exact values.
// For a mirror point (kind 1) `phi` is the azimuth of its pair's first point.
double trig_factor(int k, double phi, int kind)
{
    const int ak = k < 0 ? -k : k;
    if (kind == 2 || kind == 3) {
        if (k < 0) return 0.0;
        const double c = (kind == 3 && (ak & 1)) ? -1.0 : 1.0;
        return k == 0 ? 1.0 : sqrt(2.0) * c;
    }
    if (k == 0) return 1.0;
    if (k > 0) return sqrt(2.0) * cos(ak * phi);
    const double s = sqrt(2.0) * sin(ak * phi);
    return kind == 1 ? -s : s;
}

// The degree-L basis at a point of the folded rule: m_c = N_l^|k| P_l^|k|(mu) T_k(phi).
int basis2d_rule(int L, double mu, double phi, int kind, double *out)
{
    double Pn[24][24];
    norm_legendre(L, mu, Pn);
    int i = 0;
    for (int l = 0; l <= L; ++l)
        for (int k = -l; k <= l; ++k) {
            const int ak = k < 0 ? -k : k;
            if ((l + ak) % 2) continue;
            out[i++] = Pn[l][ak] * trig_factor(k, phi, kind);
        }
    return i;
}

template <typename T>
int dev_upload(kitrt_mn *mn, T **dst, const std::vector<T> &src)
{
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    if (cudaMalloc((void **)dst, bytes) != cudaSuccess) return KITRT_ENOMEM;
    mn->allocs.push_back(*dst);
    if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T),
                                   cudaMemcpyHostToDevice) != cudaSuccess)
        return KITRT_ECUDA;
    return KITRT_OK;
}

template <typename T>
int dev_alloc(kitrt_mn *mn, T **dst, size_t count)
{
    if (cudaMalloc((void **)dst, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess)
        return KITRT_ENOMEM;
    mn->allocs.push_back(*dst);
    return KITRT_OK;
}

}  // namespace

LaunchScope::LaunchScope(kitrt_mn *m, int k, cudaStream_t st, int64_t units) : mn(m), kind(k), s(st)
{
    ++mn->launch_count;
    if (!mn->prof_on) return;
    mn->prof_launches[k] += 1;
    mn->prof_units[k] += units;
    if (mn->prof_used >= 65536) return;
    if (mn->prof_used == mn->prof_recs.size()) {
        ProfRec r{};
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
        mn->prof_recs.push_back(r);
    }
    rec = &mn->prof_recs[mn->prof_used++];
    rec->kind = k;
    cudaEventRecord(rec->a, s);
}

LaunchScope::~LaunchScope()
{
    if (rec) cudaEventRecord(rec->b, s);
}

static const char *kProfNames[PK_COUNT] = {"closure_begin", "closure_eval_fp64", "closure_finish",
                                           "flux_update", "closure_eval_mixed", "mlp",
                                           "adjoint", "other", "closure_newton", "sn_step",
                                           "reconstruct"};

Tables kitrt_mn::tables() const
{
    Tables T;
    T.n = n;
    T.n2 = n2;
    T.Qf = Qf;
    T.Qp = Qp;
    T.m0 = 1.0 / sqrt(4.0 * kPi);
    T.rm0 = sqrt(4.0 * kPi);
    T.Mt = d_Mt;
    T.w = d_w;
    T.wox = d_wox;
    T.woy = d_woy;
    T.mbar = d_mbar;
    T.gstart = d_gstart;
    T.gidx = d_gidx;
    T.gcoef = d_gcoef;
    T.gcoef32 = d_gcoef32;
    T.Mt32 = d_Mt32;
    T.w32 = d_w32;
    T.wox32 = d_wox32;
    T.woy32 = d_woy32;
    T.mbar32 = d_mbar32;
    T.exptab = d_exptab;
    T.R = R;
    T.P = P;
    T.npair = Qf / 2;
    T.ptrig = d_ptrig;
    T.ringP = d_ringP;
    T.ringWP = d_ringWP;
    return T;
}

extern "C" {

const char *kitrt_status_string(int32_t code)
{
    switch (code) {
    case KITRT_OK: return "ok";
    case KITRT_EINVAL: return "invalid argument";
    case KITRT_ENOTREALIZABLE: return "moment vector not realizable (non-finite closure)";
    case KITRT_ENOCONVERGE: return "Newton iteration limit reached";
    case KITRT_ECHOL: return "Hessian not positive definite (Cholesky breakdown)";
    case KITRT_ELINESEARCH: return "line search exhausted";
    case KITRT_ECUDA: return "CUDA runtime error";
    case KITRT_ENOMEM: return "device allocation failed";
    case KITRT_ETIMEOUT: return "bounded device wait expired";
    case KITRT_ESCRATCH: return "batch exceeds the fixed scratch of kitrt_closure_noalloc";
    default: return "unknown status";
    }
}

int32_t kitrt_default_params(kitrt_mn_params *p)
{
    if (!p) return KITRT_EINVAL;
    memset(p, 0, sizeof(*p));
    p->degree = 2;
    p->quad_order = 10;
    p->mode = KITRT_FP64;
    p->bc = KITRT_BC_NEUMANN;
    p->tau = 1e-10;
    p->max_iter = 100;
    p->max_halvings = 30;
    p->armijo_c1 = 1e-4;
    p->polish = 1;
    p->cfl = 0.4;
    p->fallback_tol = 1e-6;
    p->order = 1;
    p->reg_gamma = 0.0;
    p->reg_keep_mass = 1;
    return KITRT_OK;
}

int32_t kitrt_mesh_create(const double *xy, int32_t nverts, const int32_t *tri, int32_t ntri,
                          kitrt_mesh **out)
{
    if (!xy || !tri || !out || nverts < 3 || ntri < 1) return KITRT_EINVAL;
    *out = nullptr;
    kitrt_mesh *m = new kitrt_mesh();
    m->C = ntri;
    cudaGetDevice(&m->device);
    m->area.resize(ntri);
    m->perim.resize(ntri);
    m->cen.resize(2 * (size_t)ntri);
    m->nrm.resize(6 * (size_t)ntri);
    m->nbr.assign(3 * (size_t)ntri, -1);
    m->r.resize(6 * (size_t)ntri);
    std::unordered_map<uint64_t, int64_t> open_edge;  // edge key -> cell*3+face
    open_edge.reserve((size_t)ntri * 2);
    double minr = 1e300;
    int rc = KITRT_OK;
    for (int32_t c = 0; c < ntri && rc == KITRT_OK; ++c) {
        int32_t v0 = tri[3 * c], v1 = tri[3 * c + 1], v2 = tri[3 * c + 2];
        if (v0 < 0 || v1 < 0 || v2 < 0 || v0 >= nverts || v1 >= nverts || v2 >= nverts) {
            rc = KITRT_EINVAL;
            break;
        }
        double ax = xy[2 * v0], ay = xy[2 * v0 + 1];
        double cross = (xy[2 * v1] - ax) * (xy[2 * v2 + 1] - ay) - (xy[2 * v2] - ax) * (xy[2 * v1 + 1] - ay);
        if (cross < 0) std::swap(v1, v2);
        cross = fabs(cross);
        if (!(cross > 0.0)) {
            rc = KITRT_EINVAL;
            break;
        }
        int32_t v[3] = {v0, v1, v2};
        m->area[c] = 0.5 * cross;
        m->cen[2 * c] = (xy[2 * v0] + xy[2 * v1] + xy[2 * v2]) / 3.0;
        m->cen[2 * c + 1] = (xy[2 * v0 + 1] + xy[2 * v1 + 1] + xy[2 * v2 + 1]) / 3.0;
        double per = 0.0;
        for (int k = 0; k < 3; ++k) {
            int32_t a = v[k], b = v[(k + 1) % 3];
            double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
            // centroid to face midpoint (second-order reconstruction)
            m->r[6 * (size_t)c + 2 * k] = 0.5 * (xy[2 * a] + xy[2 * b]) - m->cen[2 * c];
            m->r[6 * (size_t)c + 2 * k + 1] = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]) - m->cen[2 * c + 1];
            // outward normal of edge a->b of a counter-clockwise triangle, |n| = edge length
            m->nrm[6 * (size_t)c + 2 * k] = xy[2 * b + 1] - xy[2 * a + 1];
            m->nrm[6 * (size_t)c + 2 * k + 1] = xy[2 * a] - xy[2 * b];
            per += sqrt(dx * dx + dy * dy);
            uint64_t lo = (uint64_t)std::min(a, b), hi = (uint64_t)std::max(a, b);
            uint64_t key = (lo << 32) | hi;
            auto it = open_edge.find(key);
            if (it == open_edge.end()) {
                open_edge.emplace(key, (int64_t)c * 3 + k);
            } else {
                int64_t other = it->second;
                if (other < 0) {
                    rc = KITRT_EINVAL;  // third cell on one edge
                    break;
                }
                int32_t oc = (int32_t)(other / 3), ok = (int32_t)(other % 3);
                m->nbr[3 * (size_t)c + k] = oc;
                m->nbr[3 * (size_t)oc + ok] = c;
                it->second = -1;
            }
        }
        m->perim[c] = per;
        minr = std::min(minr, 2.0 * m->area[c] / per);
    }
    if (rc != KITRT_OK) {
        delete m;
        return rc;
    }
    m->min_inradius = minr;
    // .w packs, for each face k, the neighbour's index of the shared face (2 bits at 2k)
    std::vector<int4> nb4(ntri);
    for (int32_t c = 0; c < ntri; ++c) {
        int packed = 0;
        for (int k = 0; k < 3; ++k) {
            const int j = m->nbr[3 * c + k];
            if (j < 0) continue;
            for (int t = 0; t < 3; ++t)
                if (m->nbr[3 * (size_t)j + t] == c) packed |= t << (2 * k);
        }
        nb4[c] = make_int4(m->nbr[3 * c], m->nbr[3 * c + 1], m->nbr[3 * c + 2], packed);
    }
    std::vector<double> hpa(ntri);
    std::vector<float> nrm32(6 * (size_t)ntri), inva32(ntri), r32(6 * (size_t)ntri);
    std::vector<double> inva(ntri);
    for (int32_t c = 0; c < ntri; ++c) {
        hpa[c] = m->perim[c] / (2.0 * m->area[c]);
        inva[c] = 1.0 / m->area[c];
        inva32[c] = (float)(1.0 / m->area[c]);
        for (int k = 0; k < 6; ++k) {
            nrm32[6 * (size_t)c + k] = (float)m->nrm[6 * (size_t)c + k];
            r32[6 * (size_t)c + k] = (float)m->r[6 * (size_t)c + k];
        }
    }
    bool ok = cudaMalloc(&m->d_nbr, sizeof(int4) * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_nrm, sizeof(double) * 6 * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_area, sizeof(double) * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_hpa, sizeof(double) * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_nrm32, sizeof(float) * 6 * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_inva32, sizeof(float) * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_inva, sizeof(double) * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_r, sizeof(double) * 6 * ntri) == cudaSuccess &&
              cudaMalloc(&m->d_r32, sizeof(float) * 6 * ntri) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_inva, inva.data(), sizeof(double) * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_r, m->r.data(), sizeof(double) * 6 * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_r32, r32.data(), sizeof(float) * 6 * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_nrm32, nrm32.data(), sizeof(float) * 6 * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_inva32, inva32.data(), sizeof(float) * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_hpa, hpa.data(), sizeof(double) * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_nbr, nb4.data(), sizeof(int4) * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_nrm, m->nrm.data(), sizeof(double) * 6 * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(m->d_area, m->area.data(), sizeof(double) * ntri, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        kitrt_mesh_destroy(m);
        return KITRT_ENOMEM;
    }
    *out = m;
    return KITRT_OK;
}

int32_t kitrt_mesh_destroy(kitrt_mesh *m)
{
    if (!m) return KITRT_EINVAL;
    cudaFree(m->d_nbr);
    cudaFree(m->d_nrm);
    cudaFree(m->d_area);
    cudaFree(m->d_hpa);
    cudaFree(m->d_nrm32);
    cudaFree(m->d_inva32);
    cudaFree(m->d_inva);
    cudaFree(m->d_r);
    cudaFree(m->d_r32);
    delete m;
    return KITRT_OK;
}

int32_t kitrt_mesh_geometry(const kitrt_mesh *m, int32_t *ncells, double *min_inradius,
                            double *area, double *perim, double *centroid, int32_t *nbr,
                            double *nrm)
{
    if (!m) return KITRT_EINVAL;
    size_t C = m->C;
    if (ncells) *ncells = m->C;
    if (min_inradius) *min_inradius = m->min_inradius;
    if (area) memcpy(area, m->area.data(), C * sizeof(double));
    if (perim) memcpy(perim, m->perim.data(), C * sizeof(double));
    if (centroid) memcpy(centroid, m->cen.data(), 2 * C * sizeof(double));
    if (nbr) memcpy(nbr, m->nbr.data(), 3 * C * sizeof(int32_t));
    if (nrm) memcpy(nrm, m->nrm.data(), 6 * C * sizeof(double));
    return KITRT_OK;
}

int32_t kitrt_mn_destroy(kitrt_mn *mn)
{
    if (!mn) return KITRT_EINVAL;
    for (ProfRec &r : mn->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (void *p : mn->allocs) cudaFree(p);
    if (mn->h_cnt) cudaFreeHost(mn->h_cnt);
    if (mn->h_sn_flag) cudaFreeHost(mn->h_sn_flag);
    if (mn->h_check) cudaFreeHost(mn->h_check);
    if (mn->d_adj) cudaFree(mn->d_adj);
    delete mn;
    return KITRT_OK;
}

int32_t kitrt_mn_init(const kitrt_mesh *mesh, const kitrt_mn_params *params, kitrt_mn **out)
{
    if (!mesh || !params || !out) return KITRT_EINVAL;
    *out = nullptr;
    const kitrt_mn_params &p = *params;
    if (p.degree < 1 || p.degree > KITRT_MAX_DEGREE || p.quad_order < p.degree + 1 ||
        p.quad_order > 64 || !(p.tau > 0) || p.max_iter < 1 || p.max_halvings < 0 ||
        p.mode < KITRT_FP64 || p.mode > KITRT_LEARNED || (p.bc != 0 && p.bc != 1) ||
        (p.order != 1 && p.order != 2) || !(p.reg_gamma >= 0.0) ||
        (p.reg_gamma > 0.0 && p.mode == KITRT_LEARNED))
        return KITRT_EINVAL;
    kitrt_mn *mn = new kitrt_mn();
    mn->mesh = mesh;
    mn->p = p;
    mn->N = p.degree;
    mn->n = nmom_of(p.degree);
    mn->n2 = nmom_of(2 * p.degree);
    mn->npairs = mn->n * (mn->n + 1) / 2;
    mn->Q = 2 * p.quad_order * p.quad_order;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mn->nsm, cudaDevAttrMultiProcessorCount, dev);
    int rc;
#define TRY(x)                    \
    do {                          \
        rc = (x);                 \
        if (rc != KITRT_OK) {     \
            kitrt_mn_destroy(mn); \
            return rc;            \
        }                         \
    } while (0)

    // folded quadrature and tables
    FoldedRule r = folded_rule(p.quad_order);
    mn->Qf = (int)r.w.size();
    mn->Qp = (mn->Qf + 31) / 32 * 32;
    const int n = mn->n, n2 = mn->n2, Qp = mn->Qp, Qf = mn->Qf;
    std::vector<double> Mt((size_t)n2 * Qp, 0.0), w(Qp, 0.0), wox(Qp, 0.0), woy(Qp, 0.0);
    mn->h_w.resize(Qf);
    mn->h_ox.resize(Qf);
    mn->h_oy.resize(Qf);
    mn->h_M.resize((size_t)Qf * n);
    std::vector<double> mb(n, 0.0);
    double tmp[128];
    for (int q = 0; q < Qf; ++q) {
        double s = sqrt(1.0 - r.mu[q] * r.mu[q]);
        // sin(phi), cos(phi) with the pairs' exact symmetries (a mirror point uses the azimuth
        // of its pair's first point, the one before it)
        const double phi0 = r.kind[q] == 1 ? r.phi[q - 1] : r.phi[q];
        double sp, cp;
        if (r.kind[q] == 2) {
            sp = 0.0, cp = 1.0;
        } else if (r.kind[q] == 3) {
            sp = 0.0, cp = -1.0;
        } else {
            sp = r.kind[q] == 1 ? -sin(phi0) : sin(phi0);
            cp = cos(phi0);
        }
        double ox = s * sp, oy = s * cp;
        basis2d_rule(2 * mn->N, r.mu[q], phi0, r.kind[q], tmp);
        for (int c = 0; c < n2; ++c) Mt[(size_t)c * Qp + q] = tmp[c];
        for (int a = 0; a < n; ++a) mn->h_M[(size_t)q * n + a] = tmp[a];
        w[q] = r.w[q];
        wox[q] = r.w[q] * ox;
        woy[q] = r.w[q] * oy;
        mn->h_w[q] = r.w[q];
        mn->h_ox[q] = ox;
        mn->h_oy[q] = oy;
        for (int a = 0; a < n; ++a) mb[a] += r.w[q] * tmp[a];
    }
    // Gaunt coefficients G[(a,b),c] = <m_a m_b m~_c> on a rule exact for degree 4N
    FoldedRule g = folded_rule(2 * mn->N + 2);
    std::vector<double> G((size_t)mn->npairs * n2, 0.0);
    for (size_t q = 0; q < g.w.size(); ++q) {
        basis2d(2 * mn->N, g.mu[q], g.phi[q], tmp);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b <= a; ++b) {
                double ab = g.w[q] * tmp[a] * tmp[b];
                double *row = &G[(size_t)(a * (a + 1) / 2 + b) * n2];
                for (int c = 0; c < n2; ++c) row[c] += ab * tmp[c];
            }
    }
    std::vector<int32_t> gstart(mn->npairs + 1, 0), gidx;
    std::vector<double> gcoef;
    for (int pp = 0; pp < mn->npairs; ++pp) {
        gstart[pp] = (int32_t)gidx.size();
        for (int c = 0; c < n2; ++c) {
            double v = G[(size_t)pp * n2 + c];
            if (fabs(v) > 1e-12) {
                gidx.push_back(c);
                gcoef.push_back(v);
            }
        }
    }
    gstart[mn->npairs] = (int32_t)gidx.size();
    mn->gaunt_nnz = (int)gidx.size();
    std::vector<float> Mt32(Mt.begin(), Mt.end()), w32(w.begin(), w.end());
    std::vector<float> wox32(wox.begin(), wox.end()), woy32(woy.begin(), woy.end());
    // tensor-core operand of the mixed modes: the degree N+1..2N basis functions (rows n..n2-1
    // of Mt), padded to a multiple of 16 rows and split into a high and a low part in TF32
    // (nearest, ties away) and in BF16 (nearest even): [2][NP x Qp], high part first
    const int nhi = n2 - n, NP = (nhi + 15) / 16 * 16;
    std::vector<float> Mhi32((size_t)2 * NP * Qp, 0.0f);
    std::vector<unsigned short> Mhi16((size_t)2 * NP * Qp, 0);
    auto tf32 = [](float f) {
        uint32_t bits;
        memcpy(&bits, &f, 4);
        bits = (bits + 0x1000u) & ~0x1FFFu;
        float r;
        memcpy(&r, &bits, 4);
        return r;
    };
    auto bf16 = [](float f, float *back) {
        uint32_t bits;
        memcpy(&bits, &f, 4);
        const uint32_t rb = (bits + 0x7FFFu + ((bits >> 16) & 1u)) & 0xFFFF0000u;
        memcpy(back, &rb, 4);
        return (unsigned short)(rb >> 16);
    };
    for (int c = 0; c < nhi; ++c)
        for (int q = 0; q < Qp; ++q) {
            // the quadrature weight is folded into the table: the tensor cores take exp(alpha.m)
            const double x = w[q] * Mt[(size_t)(n + c) * Qp + q];
            const float hi = tf32((float)x);
            Mhi32[(size_t)c * Qp + q] = hi;
            Mhi32[((size_t)NP + c) * Qp + q] = tf32((float)(x - (double)hi));
            float bhi;
            Mhi16[(size_t)c * Qp + q] = bf16((float)x, &bhi);
            float dummy;
            Mhi16[((size_t)NP + c) * Qp + q] = bf16((float)(x - (double)bhi), &dummy);
        }
    TRY(dev_upload(mn, &mn->d_Mt, Mt));
    TRY(dev_upload(mn, &mn->d_w, w));
    TRY(dev_upload(mn, &mn->d_wox, wox));
    TRY(dev_upload(mn, &mn->d_woy, woy));
    TRY(dev_upload(mn, &mn->d_mbar, mb));
    TRY(dev_upload(mn, &mn->d_mbar32, std::vector<float>(mb.begin(), mb.end())));
    TRY(dev_upload(mn, &mn->d_gstart, gstart));
    TRY(dev_upload(mn, &mn->d_gidx, gidx));
    TRY(dev_upload(mn, &mn->d_gcoef, gcoef));
    TRY(dev_upload(mn, &mn->d_gcoef32, std::vector<float>(gcoef.begin(), gcoef.end())));
    TRY(dev_upload(mn, &mn->d_Mt32, Mt32));
    TRY(dev_upload(mn, &mn->d_w32, w32));
    TRY(dev_upload(mn, &mn->d_wox32, wox32));
    TRY(dev_upload(mn, &mn->d_woy32, woy32));
    // unweighted folded directions for the S_N step (0 on padding)
    std::vector<double> oxp(Qp, 0.0), oyp(Qp, 0.0);
    for (int q = 0; q < Qf; ++q) {
        oxp[q] = mn->h_ox[q];
        oyp[q] = mn->h_oy[q];
    }
    std::vector<float> oxp32(oxp.begin(), oxp.end()), oyp32(oyp.begin(), oyp.end());
    TRY(dev_upload(mn, &mn->d_ox, oxp));
    TRY(dev_upload(mn, &mn->d_oy, oyp));
    TRY(dev_upload(mn, &mn->d_ox32, oxp32));
    TRY(dev_upload(mn, &mn->d_oy32, oyp32));
    // 2^(j/2048), j = 0..2047, then 2^(j/2048) ln2/2048 (kexp_scaled), rounded to double from
    // extended precision
    std::vector<double> exptab(4096);
    for (int j = 0; j < 2048; ++j) {
        const long double t = exp2l((long double)j / 2048.0L);
        exptab[j] = (double)t;
        exptab[2048 + j] = (double)(t * (logl(2.0L) / 2048.0L));
    }
    TRY(dev_upload(mn, &mn->d_exptab, exptab));
    // sum-factorised sweeps: azimuthal factors per pair and Legendre factors per ring
    {
        const int L2 = 2 * mn->N, TW = 2 * L2 + 1;
        mn->R = (int)r.ring_mu.size();
        mn->P = r.P;
        std::vector<double> ptrig((size_t)(Qp / 2) * TW, 0.0);
        for (int pr = 0; pr < Qf / 2; ++pr) {
            const int q = 2 * pr;
            const bool zero_pi = r.kind[q] == 2;
            for (int k = 0; k <= L2; ++k)
                ptrig[(size_t)pr * TW + k] = trig_factor(k, r.phi[q], zero_pi ? 2 : 0);
            for (int k = 1; k <= L2; ++k)
                ptrig[(size_t)pr * TW + L2 + k] =
                    zero_pi ? trig_factor(k, r.phi[q], 3) : trig_factor(-k, r.phi[q], 0);
        }
        std::vector<double> ringP((size_t)(mn->R + 1) * n2, 0.0), ringWP((size_t)(mn->R + 1) * n2, 0.0);
        for (int rg = 0; rg < mn->R; ++rg) {
            double Pn[24][24];
            norm_legendre(2 * mn->N, r.ring_mu[rg], Pn);
            int c = 0;
            for (int l = 0; l <= 2 * mn->N; ++l)
                for (int k = -l; k <= l; k += 2, ++c) {
                    ringP[(size_t)rg * n2 + c] = Pn[l][k < 0 ? -k : k];
                    ringWP[(size_t)rg * n2 + c] = r.ring_w[rg] * Pn[l][k < 0 ? -k : k];
                }
        }
        TRY(dev_upload(mn, &mn->d_ptrig, ptrig));
        TRY(dev_upload(mn, &mn->d_ringP, ringP));
        TRY(dev_upload(mn, &mn->d_ringWP, ringWP));
    }
    TRY(dev_upload(mn, &mn->d_Mhi32, Mhi32));
    TRY(dev_upload(mn, &mn->d_Mhi16, Mhi16));

    // workspace
    const size_t C = mesh->C;
    NewtonState &S = mn->st;
    TRY(dev_alloc(mn, &S.alpha, C * n));
    TRY(dev_alloc(mn, &S.dir, C * n));
    TRY(dev_alloc(mn, &S.U, C * n));
    TRY(dev_alloc(mn, &S.fsum, C));
    TRY(dev_alloc(mn, &S.f0, C));
    TRY(dev_alloc(mn, &S.gd, C));
    TRY(dev_alloc(mn, &S.L, C * mn->npairs));
    TRY(dev_alloc(mn, &S.lam, C));
    TRY(dev_alloc(mn, &S.phase, C));
    TRY(dev_alloc(mn, &S.iters, C));
    TRY(dev_alloc(mn, &S.halv, C));
    TRY(dev_alloc(mn, &S.evals, C));
    TRY(dev_alloc(mn, &S.status, C));
    TRY(dev_alloc(mn, &S.list[0], C));
    TRY(dev_alloc(mn, &S.list[1], C));
    TRY(dev_alloc(mn, &S.cnt, 16));
    // no cell has a closure state yet: NaN alphas never equal a caller's alpha bit for bit, so the
    // first kitrt_step starts every cell from its given alpha
    if (cudaMemset(S.alpha, 0xff, sizeof(double) * C * n) != cudaSuccess ||
        cudaMemset(S.dir, 0, sizeof(double) * C * n) != cudaSuccess ||
        cudaMemset(S.status, 0xff, sizeof(int32_t) * C) != cudaSuccess) {
        kitrt_mn_destroy(mn);
        return KITRT_ECUDA;
    }
    TRY(dev_alloc(mn, &mn->d_psi, C * Qp));
    // the padding points of psi are never written (their weight is 0): zeros keep them finite
    if (cudaMemset(mn->d_psi, 0, sizeof(double) * C * Qp) != cudaSuccess) {
        kitrt_mn_destroy(mn);
        return KITRT_ECUDA;
    }
    // sweep work split (sweep.cuh): both sweeps run persistent grids of the CTAs that fit on the
    // SMs at once and split the quadrature of each tile so that every CTA gets several work items
    // (4 for the tensor-core sweep, 2 for the FP64 sweep). A split never needs more than
    // C + target * 128 columns per moment.
    mn->grid_mixed = p.mode == KITRT_FP64 ? mn->nsm : mixed_sweep_grid(mn);
    mn->target_mixed = 4 * mn->grid_mixed;
    mn->grid_fp64 = fp64_sweep_grid(mn);
    mn->target_fp64 = 2 * mn->grid_fp64;
    mn->vs = (int)C + 128 * std::max(mn->target_mixed, mn->target_fp64) + 128;
    TRY(dev_alloc(mn, &mn->d_Vacc, (size_t)mn->vs * n2));
    if (cudaMemset(mn->d_Vacc, 0, sizeof(double) * (size_t)mn->vs * n2) != cudaSuccess) {
        kitrt_mn_destroy(mn);
        return KITRT_ECUDA;
    }
    if (p.mode != KITRT_FP64) {
        TRY(dev_alloc(mn, &mn->d_psi32, C * Qp));
        if (cudaMemset(mn->d_psi32, 0, sizeof(float) * C * Qp) != cudaSuccess) {
            kitrt_mn_destroy(mn);
            return KITRT_ECUDA;
        }
        TRY(dev_alloc(mn, &mn->d_zero32, (size_t)Qp));
        if (cudaMemset(mn->d_zero32, 0, sizeof(float) * Qp) != cudaSuccess) {
            kitrt_mn_destroy(mn);
            return KITRT_ECUDA;
        }
        if (p.mode == KITRT_LEARNED) TRY(dev_alloc(mn, &mn->d_alpha_nn, C * (size_t)n));
        TRY(dev_alloc(mn, &S.h64, C));
        TRY(dev_alloc(mn, &S.gnorm, C));
        if (p.mode == KITRT_LEARNED) {
            TRY(dev_alloc(mn, &S.lfac, C));
            if (cudaMemset(S.lfac, 0, sizeof(int32_t) * C) != cudaSuccess) {
                kitrt_mn_destroy(mn);
                return KITRT_ECUDA;
            }
        }
    }
    if (cudaMallocHost(&mn->h_cnt, 16 * sizeof(int32_t)) != cudaSuccess) {
        kitrt_mn_destroy(mn);
        return KITRT_ENOMEM;
    }
    TRY(dev_alloc(mn, &mn->d_sn_flag, 1));
    {
        double *cellc = nullptr;
        TRY(dev_alloc(mn, &cellc, C * 12));
        mn->d_sn_cell = cellc;
    }
    if (p.order == 2) {
        TRY(dev_alloc(mn, &mn->d_ustage, C * n));
        if (p.mode == KITRT_FP64) {
            double *pf = nullptr;
            TRY(dev_alloc(mn, &pf, C * 3 * Qp));
            mn->d_psif = pf;
        } else {
            float *pf = nullptr;
            TRY(dev_alloc(mn, &pf, C * 3 * Qp));
            mn->d_psif = pf;
        }
    }
    TRY(dev_alloc(mn, &mn->d_check, 2));
    if (cudaMallocHost(&mn->h_check, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        kitrt_mn_destroy(mn);
        return KITRT_ENOMEM;
    }
    if (cudaMallocHost(&mn->h_sn_flag, sizeof(int32_t)) != cudaSuccess) {
        kitrt_mn_destroy(mn);
        return KITRT_ENOMEM;
    }
#undef TRY
    *out = mn;
    return KITRT_OK;
}

int32_t kitrt_mn_sizes(const kitrt_mn *mn, int32_t *nmom, int32_t *nquad, int32_t *nquad_folded)
{
    if (!mn) return KITRT_EINVAL;
    if (nmom) *nmom = mn->n;
    if (nquad) *nquad = mn->Q;
    if (nquad_folded) *nquad_folded = mn->Qf;
    return KITRT_OK;
}

int32_t kitrt_mn_work(const kitrt_mn *mn, kitrt_work *out)
{
    if (!mn || !out) return KITRT_EINVAL;
    const double n = mn->n, n2 = mn->n2, Qf = mn->Qf, N = mn->N;
    const bool fp64 = mn->p.mode == KITRT_FP64;
    out->nmom = mn->n;
    out->nmom2 = mn->n2;
    out->nquad_folded = mn->Qf;
    out->gaunt_nnz = mn->gaunt_nnz;
    // sum-factorised sweep (sweep.cuh), per pair of points: exponent C (N FMA) and S (1 MUL +
    // N-1 FMA), z = C +- S (2), e +- e' (2), azimuthal sums up to degree L (1 ADD + 2L FMA);
    // per ring: the exponent coefficients (n FMA) and the moments (nmom(L) FMA). FMA = 2 flops.
    const double L = fp64 ? 2 * N : N, nout = fp64 ? n2 : n;
    const double pairs = Qf / 2, rings = mn->R;
    const double pair_ops = N + N + 2 + 2 + 1 + 2 * L, pair_fmas = N + (N - 1) + 2 * L;
    const double ring_fmas = n + nout;
    out->sweep_fp64_flops = pairs * (pair_ops + pair_fmas) + rings * 2 * ring_fmas;
    out->sweep_fp64_ops = pairs * pair_ops + rings * ring_fmas + Qf * (fp64 ? kExpFp64Ops : kExpScaledFp64Ops);
    out->exps = Qf;
    out->tensor_flops = fp64 ? 0.0 : 3.0 * 2.0 * (n2 - n) * Qf;
    out->newton_flops = 2.0 * mn->gaunt_nnz + n * n * n / 3 + 2 * n * n;
    out->sweep_grid = fp64 ? mn->grid_fp64 : mn->grid_mixed;
    out->sweep_items = fp64 ? mn->target_fp64 : mn->target_mixed;
    return KITRT_OK;
}

int32_t kitrt_mn_quadrature(const kitrt_mn *mn, double *w, double *omega, double *m)
{
    if (!mn) return KITRT_EINVAL;
    for (int q = 0; q < mn->Qf; ++q) {
        if (w) w[q] = mn->h_w[q];
        if (omega) {
            omega[2 * q] = mn->h_ox[q];
            omega[2 * q + 1] = mn->h_oy[q];
        }
    }
    if (m) memcpy(m, mn->h_M.data(), sizeof(double) * mn->h_M.size());
    return KITRT_OK;
}

int32_t kitrt_isotropic_alpha(kitrt_mn *mn, const double *u, double *alpha, void *stream)
{
    if (!mn || !u || !alpha) return KITRT_EINVAL;
    return launch_isotropic(mn->tables(), mn->mesh->C, u, alpha, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Newton driver (shared by kitrt_closure and kitrt_step)
// ------------------------------------------------------------------------------------------

// The polish step (one more full Newton step once the test passes) needs the exact Hessian: it
// is applied in FP64 mode only.
static int polish_of(const kitrt_mn *mn) { return mn->p.polish && mn->p.mode == KITRT_FP64; }

// Runs the closure of cells 0..C-1 to completion. first = 1 starts from alpha_in (evaluation
// first); first = 0 reuses the state of the previous closure as the predictor. In the learned
// mode the network proposes alpha for every cell that needs a closure, and only the cells whose
// FP64 residual test fails enter the Newton sweeps. Leaves the converged state in mn->st; returns
// the first failure status or KITRT_OK.
static int run_closure(kitrt_mn *mn, int C, const double *u, const double *alpha_in, int first,
                       cudaStream_t s, kitrt_stats *stats, float *psi32 = nullptr)
{
    const Tables T = mn->tables();
    NewtonParams np{mn->p.tau, mn->p.armijo_c1, mn->p.max_iter, mn->p.max_halvings, polish_of(mn),
                    mn->p.reg_gamma, mn->p.reg_keep_mass ? 1 : 0};
    const bool learned = mn->p.mode == KITRT_LEARNED;
    if (learned && !mn->has_mlp) return KITRT_EINVAL;
    CUDA_OK(cudaMemsetAsync(mn->st.cnt, 0, 16 * sizeof(int32_t), s));
    int rc = launch_begin(mn, T, mn->st, C, u, alpha_in, first, np, s, learned);
    if (rc) return rc;
    if (learned) {
        rc = launch_mlp_infer(mn, u, mn->st.list[1], mn->st.cnt + 8, C, mn->d_alpha_nn, s);
        if (!rc) rc = launch_learned_pass(mn, T, mn->st, C, u, psi32, first == 1, s);
        if (rc) return rc;
    }
    // rounds are launched in batches between two reads of the counters; the first batch is as long
    // as the previous closure needed (its largest evaluation count), so that a steady run launches
    // no empty round and synchronises once
    const int max_launch = (mn->p.max_iter + 1) * (mn->p.max_halvings + 1) + 1;
    int k = 0;
    for (int batch = mn->pass_hint;; batch = 4) {
        for (int b = 0; b < batch; ++b, ++k) {
            // quadrature sweeps write each listed cell's moment row; the thread-per-cell Newton
            // step then takes every listed cell
            if (mn->p.mode == KITRT_FP64) {
                rc = launch_eval_fp64(mn, T, mn->st, C, u, k, np, s, false, nullptr, mn->d_Vacc);
            } else {
                // FP64 sweep of the cells handed over in earlier rounds (none in the first: the
                // closure starts with every hand-over cleared), then the tensor-core sweep of the
                // others (cells handed over now wait for the next round, so no cell is evaluated
                // twice in one round)
                if (k > 0) rc = launch_eval_fp64(mn, T, mn->st, C, u, k, np, s, true, psi32, mn->d_Vacc);
                if (!rc) rc = launch_eval_mixed(mn, T, mn->st, C, u, k, np, s, psi32);
            }
            if (!rc) rc = launch_sum_parts(mn, mn->st, k, mn->d_Vacc, s);
            if (!rc) rc = launch_post(mn, T, mn->st, C, u, k, np, mn->d_Vacc, s);
            if (rc) return rc;
        }
        CUDA_OK(cudaMemcpyAsync(mn->h_cnt, mn->st.cnt, 12 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
        if (mn->h_cnt[7]) return mn->h_cnt[7];
        int active = mn->h_cnt[k % 3];
        if (active == 0) break;
        if (k >= max_launch) return KITRT_ETIMEOUT;
    }
    mn->pass_hint = std::max(1, std::min(8, (int)mn->h_cnt[4]));
    // the sweeps' evaluations (the network's residual passes run in their own kernel)
    if (mn->prof_on) mn->prof_units[mn->p.mode == KITRT_FP64 ? PK_EVAL : PK_EVAL_MIXED] += mn->h_cnt[6];
    if (mn->prof_on && mn->p.mode == KITRT_LEARNED) mn->prof_units[PK_MLP] += mn->h_cnt[10];
    if (stats) {
        stats->closures += C;
        stats->evaluations += mn->h_cnt[6] + mn->h_cnt[10];
        stats->max_evals = std::max(stats->max_evals, mn->h_cnt[4]);
        stats->failed = mn->h_cnt[3];
        stats->fallbacks += mn->h_cnt[5];
        stats->restarts += mn->h_cnt[9];
        if (mn->p.mode == KITRT_LEARNED) stats->proposals += mn->h_cnt[8];
        stats->handovers += mn->h_cnt[11];
    }
    if (mn->h_cnt[3] > 0) {
        // report the first failing code
        std::vector<int32_t> stv(C);
        CUDA_OK(cudaMemcpy(stv.data(), mn->st.status, sizeof(int32_t) * C, cudaMemcpyDeviceToHost));
        for (int32_t v : stv)
            if (v) return v;
    }
    return KITRT_OK;
}

extern "C" {

}  // extern "C"

// One FP64 step on device buffers without statistics (used by the adjoint): closure of u (from
// alpha when first, else from the previous closure's state), final alpha into `alpha`, ansatz,
// flux and update of u.
int kitrt_internal_step(kitrt_mn *mn, double *u, double *alpha, const double *sa, const double *ss,
                        const double *q, double dt, int first, cudaStream_t s)
{
    const int C = mn->mesh->C;
    int rc = run_closure(mn, C, u, alpha, first, s, nullptr);
    if (rc) return rc;
    rc = launch_finish(mn, mn->tables(), mn->st, C, alpha, mn->d_psi, nullptr, polish_of(mn), !first, s);
    if (rc) return rc;
    return launch_flux_update(mn, mn->tables(), C, mn->d_psi, nullptr, u, sa, ss, q, dt, mn->p.bc, s);
}

extern "C" {

int32_t kitrt_closure_batch(kitrt_mn *mn, const double *u, double *alpha, int32_t *status,
                            int32_t ncells, void *stream, kitrt_stats *stats)
{
    if (!mn || !u || !alpha || ncells < 0 || ncells > mn->mesh->C) return KITRT_EINVAL;
    if (ncells == 0) return KITRT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (stats) memset(stats, 0, sizeof(*stats));
    const int64_t launches0 = mn->launch_count;
    int rc = run_closure(mn, ncells, u, alpha, 1, s, stats);
    int rc2 = launch_finish(mn, mn->tables(), mn->st, ncells, alpha, nullptr, nullptr,
                            polish_of(mn), 0, s);
    if (status)
        CUDA_OK(cudaMemcpyAsync(status, mn->st.status, sizeof(int32_t) * ncells,
                                cudaMemcpyDeviceToDevice, s));
    if (stats) {
        stats->launches = mn->launch_count - launches0;
        CUDA_OK(cudaStreamSynchronize(s));
    }
    return rc ? rc : rc2;
}

int32_t kitrt_closure(kitrt_mn *mn, const double *u, double *alpha, int32_t *status,
                      void *stream, kitrt_stats *stats)
{
    if (!mn) return KITRT_EINVAL;
    return kitrt_closure_batch(mn, u, alpha, status, mn->mesh->C, stream, stats);
}

int32_t kitrt_ansatz(kitrt_mn *mn, const double *alpha, double *psi, void *stream)
{
    if (!mn || !alpha || !psi) return KITRT_EINVAL;
    return launch_ansatz(mn->tables(), mn->mesh->C, alpha, psi, (cudaStream_t)stream);
}

int32_t kitrt_step(kitrt_mn *mn, double *u, double *alpha, const double *sigma_a,
                   const double *sigma_s, const double *q, double dt, int32_t nsteps,
                   int32_t *status, void *stream, kitrt_stats *stats)
{
    if (!mn || !u || !alpha || !sigma_a || !sigma_s || !q || nsteps < 0) return KITRT_EINVAL;
    // the density of the transformed CSD equation is applied by the first-order flux only
    if (mn->d_invrho && mn->p.order != 1) return KITRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (dt <= 0.0) dt = mn->p.cfl * mn->mesh->min_inradius;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->dt = dt;
    }
    const int64_t launches0 = mn->launch_count;
    const int C = mn->mesh->C;
    const Tables T = mn->tables();
    if (nsteps == 0) return KITRT_OK;
    // first step: each cell whose given alpha is, bit for bit, the one the solver last returned
    // for it continues from the stored state of that closure (the Newton predictor starts from
    // the stored factor), every other cell from its given alpha; after kitrt_mn_reset every cell
    // starts from its given alpha. Later steps continue from the previous step's closure.
    const int first = mn->force_cold ? 1 : 2;
    mn->force_cold = false;
    // stability of the explicit step (positivity of the kinetic update at every quadrature point):
    // dt (P_i / (2 A_i) + sigma_a,i + sigma_s,i) <= 1 in every cell; the test's result is read
    // back with the first closure's completion counters, before u is touched
    int rc = check_stability(mn, sigma_a, sigma_s, dt, s, false);
    if (rc) return rc;
    for (int32_t it = 0; it < nsteps && mn->p.order == 2; ++it) {
        // Heun [Sec. 4.3]: u* = u + dt L(u), u <- (u + u* + dt L(u*)) / 2, each stage with its
        // own closure (the second continues from the first), reconstruction and flux
        const bool fp64 = mn->p.mode == KITRT_FP64;
        const void *psi = fp64 ? (const void *)mn->d_psi : (const void *)mn->d_psi32;
        for (int stage = 0; stage < 2 && !rc; ++stage) {
            double *uin = stage == 0 ? u : mn->d_ustage;
            rc = run_closure(mn, C, uin, alpha, it == 0 && stage == 0 ? first : 0, s, stats,
                             fp64 ? nullptr : mn->d_psi32);
            if (!rc && it == 0 && stage == 0) rc = stability_verdict(mn);
            if (!rc)
                rc = launch_finish(mn, T, mn->st, C, alpha, fp64 ? mn->d_psi : nullptr, nullptr,
                                   polish_of(mn), it > 0 || stage > 0, s);
            if (!rc) rc = launch_recon(mn, T, psi, mn->d_psif, !fp64, mn->p.bc, s);
            if (!rc)
                rc = stage == 0 ? launch_flux2(mn, T, psi, mn->d_psif, !fp64, u, nullptr, mn->d_ustage,
                                               sigma_a, sigma_s, q, dt, 0.0, 1.0, mn->p.bc, s)
                                : launch_flux2(mn, T, psi, mn->d_psif, !fp64, mn->d_ustage, u, u,
                                               sigma_a, sigma_s, q, dt, 0.5, 0.5, mn->p.bc, s);
        }
        if (rc) break;
    }
    for (int32_t it = 0; it < nsteps && mn->p.order == 1; ++it) {
        const bool fp64 = mn->p.mode == KITRT_FP64;
        // mixed modes: the evaluation sweeps write the FP32 ansatz of every accepted point, and
        // with no polish step the solution's ansatz is already in place
        rc = run_closure(mn, C, u, alpha, it == 0 ? first : 0, s, stats, fp64 ? nullptr : mn->d_psi32);
        if (!rc && it == 0) rc = stability_verdict(mn);
        if (rc) break;
        // compare_prev (skip psi when alpha is bitwise unchanged) only once alpha holds the
        // previous step's output, which is always the case after the first step of a call and for
        // a first step that continued every cell; a cold first step recomputes psi everywhere
        rc = launch_finish(mn, T, mn->st, C, alpha, fp64 ? mn->d_psi : nullptr, nullptr,
                           polish_of(mn), it > 0, s);
        if (rc) break;
        rc = launch_flux_update(mn, T, C, fp64 ? mn->d_psi : nullptr, fp64 ? nullptr : mn->d_psi32,
                                u, sigma_a, sigma_s, q, dt, mn->p.bc, s);
        if (rc) break;
    }
    if (status)
        CUDA_OK(cudaMemcpyAsync(status, mn->st.status, sizeof(int32_t) * C,
                                cudaMemcpyDeviceToDevice, s));
    if (stats) {
        stats->launches = mn->launch_count - launches0;
        CUDA_OK(cudaStreamSynchronize(s));
    }
    return rc;
}

int32_t kitrt_mn_reset(kitrt_mn *mn)
{
    if (!mn) return KITRT_EINVAL;
    mn->force_cold = true;
    return KITRT_OK;
}

int32_t kitrt_hessian(kitrt_mn *mn, const double *alpha, double *H, void *stream)
{
    if (!mn || !alpha || !H) return KITRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int C = mn->mesh->C;
    const Tables T = mn->tables();
    if (!mn->d_V && cudaMalloc(&mn->d_V, sizeof(double) * (size_t)C * mn->n2) != cudaSuccess)
        return KITRT_ENOMEM;
    if (mn->d_V && std::find(mn->allocs.begin(), mn->allocs.end(), (void *)mn->d_V) == mn->allocs.end())
        mn->allocs.push_back(mn->d_V);
    int rc = mn->p.mode == KITRT_FP64 ? launch_moments_fp64(mn, T, C, alpha, mn->d_V, s)
                                      : launch_moments_mixed(mn, T, C, alpha, mn->d_V, s);
    if (rc) return rc;
    return launch_gaunt(mn, T, C, mn->d_V, H, s);
}

int32_t kitrt_profile_enable(kitrt_mn *mn, int32_t on)
{
    if (!mn) return KITRT_EINVAL;
    if (on) {
        mn->prof_used = 0;
        for (int k = 0; k < PK_COUNT; ++k) mn->prof_launches[k] = mn->prof_units[k] = 0;
    }
    mn->prof_on = on != 0;
    return KITRT_OK;
}

int32_t kitrt_profile_read(kitrt_mn *mn, kitrt_profile_entry *out, int32_t max_entries,
                           int32_t *n_entries)
{
    if (!mn || (!out && max_entries > 0)) return KITRT_EINVAL;
    double ms[PK_COUNT] = {};
    for (size_t i = 0; i < mn->prof_used; ++i) {
        ProfRec &r = mn->prof_recs[i];
        CUDA_OK(cudaEventSynchronize(r.b));
        float t = 0.f;
        CUDA_OK(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.kind] += t;
    }
    int cnt = 0;
    for (int k = 0; k < PK_COUNT && cnt < max_entries; ++k) {
        if (mn->prof_launches[k] == 0) continue;
        kitrt_profile_entry &e = out[cnt++];
        memset(&e, 0, sizeof(e));
        strncpy(e.name, kProfNames[k], sizeof(e.name) - 1);
        e.launches = mn->prof_launches[k];
        e.units = mn->prof_units[k];
        e.total_ms = ms[k];
    }
    if (n_entries) *n_entries = cnt;
    return KITRT_OK;
}

}  // extern "C"
