// Mesh upload: orientation, reference geometry, block pattern (SELL-32),
// element-to-slot gather lists and boundary data (§3.1 discretization on P1
// tetrahedra; boundary conditions of eq. strong_form_dirichlet_u).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace hyel {

namespace {

struct HostGeom {
    std::vector<double> geo;  // [14][E]
};

inline double det3(const double m[3][3]) {
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

template <typename T>
T *upload(Ctx &c, const std::vector<T> &h) {
    if (h.empty()) return nullptr;
    T *d = dalloc_n<T>(c, h.size());
    HYEL_CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c.stream));
    return d;
}

}  // namespace

static void mesh_upload_impl(Ctx &c, int64_t N, const double *X, int64_t E, const int32_t *tets_in,
                             const hyel_bc *bc, const hyel_material *mat) {
    if (N < 4 || E < 1 || !X || !tets_in || !mat) fail(HYEL_EINVAL, "mesh_upload: need N >= 4, E >= 1, X, tets, mat");
    if (N > (int64_t)1 << 30 || E * kRecords >= ((int64_t)1 << 31)) fail(HYEL_EINVAL, "mesh_upload: mesh too large for int32 indices");
    if (mat->vol_model != HYEL_VOL_GIBBS && mat->vol_model != HYEL_VOL_INCOMPRESSIBLE)
        fail(HYEL_EINVAL, "mesh_upload: vol_model must be HYEL_VOL_GIBBS or HYEL_VOL_INCOMPRESSIBLE");
    if (mat->n_fibres != 0 && mat->n_fibres != 2) fail(HYEL_EINVAL, "mesh_upload: n_fibres must be 0 or 2");
    if (mat->n_fibres == 2 && (!mat->fibre_a1 || !mat->fibre_a2)) fail(HYEL_EINVAL, "mesh_upload: fibre directions required");
    if (!(mat->rho0 > 0) || !(mat->c_m >= 0)) fail(HYEL_EINVAL, "mesh_upload: rho0 must be > 0 and c_m >= 0");
    if (bc && bc->n_dirichlet > 0 && (!bc->dir_node || !bc->dir_comp)) fail(HYEL_EINVAL, "mesh_upload: Dirichlet arrays missing");
    if (bc && bc->n_traction_tris > 0 && !bc->traction_tris) fail(HYEL_EINVAL, "mesh_upload: traction triangles missing");
    if (bc && !(bc->t_ramp > 0)) fail(HYEL_EINVAL, "mesh_upload: t_ramp must be > 0");

    // release the previous mesh and everything sized by it
    free_workspace(c);
    amg_free(c);
    shat_free(c);
    acheb_free(c);
    dfree_all(c);
    c.mesh = DeviceMesh();
    c.mat = DeviceMatrix();
    c.stage = nullptr;
    c.vec = nullptr;
    c.red = nullptr;
    c.counter = nullptr;
    c.err = nullptr;

    DeviceMesh &m = c.mesh;
    m.N = N;
    m.E = E;
    m.vol_model = mat->vol_model;
    m.n_fibres = mat->n_fibres;
    m.rho0 = mat->rho0;
    m.kd = mat->kd;
    for (int i = 0; i < 3; i++) m.body[i] = mat->body[i];
    m.t_ramp = bc ? bc->t_ramp : 1.0;

    // ---- orientation and reference geometry
    std::vector<int32_t> tets(tets_in, tets_in + 4 * E);
    std::vector<double> geo(14 * (size_t)E);
    std::vector<double> mat4(4 * (size_t)E);
    std::vector<double> hmax_all((size_t)E);
    for (int64_t e = 0; e < E; e++) {
        int32_t *t = &tets[4 * e];
        for (int a = 0; a < 4; a++)
            if (t[a] < 0 || t[a] >= N) fail(HYEL_EINVAL, "mesh_upload: tet node index out of range");
        double J[3][3];  // J[I][a] = X_a - X_0
        for (int a = 0; a < 3; a++)
            for (int I = 0; I < 3; I++) J[I][a] = X[3 * (int64_t)t[a + 1] + I] - X[3 * (int64_t)t[0] + I];
        double d = det3(J);
        if (d < 0) {
            std::swap(t[1], t[2]);
            for (int I = 0; I < 3; I++) std::swap(J[I][0], J[I][1]);
            d = -d;
        }
        double hmax = 0;
        for (int a = 0; a < 4; a++)
            for (int b = a + 1; b < 4; b++) {
                double s = 0;
                for (int I = 0; I < 3; I++) {
                    double q = X[3 * (int64_t)t[b] + I] - X[3 * (int64_t)t[a] + I];
                    s += q * q;
                }
                hmax = std::max(hmax, std::sqrt(s));
            }
        if (!(d > 1e-14 * hmax * hmax * hmax)) fail(HYEL_EINVERTED, "mesh_upload: degenerate (zero-volume) tetrahedron");
        // inverse of J: Jinv[a][I] = d xi_a / d X_I
        double inv[3][3];
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
        // g[A][I] = sum_a dN_A/dxi_a * inv[a][I], dN_0/dxi = (-1,-1,-1), dN_a/dxi = e_a
        for (int I = 0; I < 3; I++) {
            double g1 = inv[0][I], g2 = inv[1][I], g3 = inv[2][I];
            geo[(0 * 3 + I) * E + e] = -(g1 + g2 + g3);
            geo[(1 * 3 + I) * E + e] = g1;
            geo[(2 * 3 + I) * E + e] = g2;
            geo[(3 * 3 + I) * E + e] = g3;
        }
        double V = d / 6.0;
        geo[12 * E + e] = V;
        double mu = mat->mu_e ? mat->mu_e[e] : mat->mu;
        double kappa = mat->kappa_e ? mat->kappa_e[e] : mat->kappa;
        double k1 = mat->k1_e ? mat->k1_e[e] : mat->k1;
        double k2 = mat->k2_e ? mat->k2_e[e] : mat->k2;
        if (!(mu > 0)) fail(HYEL_EINVAL, "mesh_upload: mu must be > 0");
        if (mat->vol_model == HYEL_VOL_GIBBS && !(kappa > 0)) fail(HYEL_EINVAL, "mesh_upload: kappa must be > 0");
        if (mat->n_fibres == 2 && !(k2 > 0)) fail(HYEL_EINVAL, "mesh_upload: k2 must be > 0");
        // tau_M = c_m h / (c rho0) (§3.1)
        double cw = mat->vol_model == HYEL_VOL_GIBBS ? std::sqrt((kappa + 4.0 * mu / 3.0) / mat->rho0)
                                                      : std::sqrt(mu / mat->rho0);
        geo[13 * E + e] = mat->c_m * hmax / (cw * mat->rho0);
        hmax_all[e] = hmax;
        mat4[0 * E + e] = mu;
        mat4[1 * E + e] = kappa;
        mat4[2 * E + e] = k1;
        mat4[3 * E + e] = k2;
    }

    // ---- node -> (element, local) lists, ascending element order
    std::vector<int32_t> node_ptr(N + 1, 0), node_list(4 * (size_t)E);
    for (int64_t e = 0; e < E; e++)
        for (int a = 0; a < 4; a++) node_ptr[tets[4 * e + a] + 1]++;
    for (int64_t i = 0; i < N; i++) node_ptr[i + 1] += node_ptr[i];
    {
        std::vector<int32_t> fill(node_ptr.begin(), node_ptr.end() - 1);
        for (int64_t e = 0; e < E; e++)
            for (int a = 0; a < 4; a++) node_list[fill[tets[4 * e + a]]++] = (int32_t)(4 * e + a);
    }
    for (int64_t i = 0; i < N; i++)
        if (node_ptr[i + 1] == node_ptr[i]) fail(HYEL_EINVAL, "mesh_upload: a node belongs to no element");

    // ---- block adjacency (CSR, ascending columns)
    std::vector<int32_t> row_ptr(N + 1, 0);
    std::vector<int32_t> cols;
    cols.reserve((size_t)N * 16);
    std::vector<int32_t> cand;
    for (int64_t i = 0; i < N; i++) {
        cand.clear();
        for (int32_t q = node_ptr[i]; q < node_ptr[i + 1]; q++) {
            int64_t e = node_list[q] / 4;
            for (int b = 0; b < 4; b++) cand.push_back(tets[4 * e + b]);
        }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        cols.insert(cols.end(), cand.begin(), cand.end());
        row_ptr[i + 1] = (int32_t)cols.size();
    }
    m.nnzb = (int64_t)cols.size();

    // ---- SELL-32 layout
    m.nslices = (int32_t)((N + 31) / 32);
    std::vector<int32_t> slice_ptr(m.nslices + 1, 0), row_len(N);
    for (int32_t s = 0; s < m.nslices; s++) {
        int32_t len = 0;
        for (int t = 0; t < 32; t++) {
            int64_t r = (int64_t)s * 32 + t;
            if (r < N) len = std::max(len, row_ptr[r + 1] - row_ptr[r]);
        }
        slice_ptr[s + 1] = slice_ptr[s] + len;
    }
    m.ncols = slice_ptr[m.nslices];
    m.nslots = m.ncols * 32;
    if (m.nslots >= ((int64_t)1 << 31) / 9) fail(HYEL_EINVAL, "mesh_upload: pattern too large");
    std::vector<int32_t> col(m.nslots, 0), diag_slot(N), mirror(m.nslots, -1);
    std::vector<int64_t> csr_slot(m.nnzb);
    auto slot_of = [&](int64_t r, int32_t j) -> int64_t { return ((int64_t)slice_ptr[r >> 5] + j) * 32 + (r & 31); };
    for (int64_t r = 0; r < N; r++) {
        int32_t len = row_ptr[r + 1] - row_ptr[r];
        row_len[r] = len;
        int32_t slen = slice_ptr[(r >> 5) + 1] - slice_ptr[r >> 5];
        for (int32_t j = 0; j < slen; j++) {
            int64_t q = slot_of(r, j);
            if (j < len) {
                col[q] = cols[row_ptr[r] + j];
                csr_slot[row_ptr[r] + j] = q;
                if (col[q] == r) diag_slot[r] = (int32_t)q;
            } else {
                col[q] = (int32_t)r;
            }
        }
    }
    auto find_slot = [&](int64_t r, int32_t cidx) -> int64_t {
        const int32_t *b = cols.data() + row_ptr[r], *e2 = cols.data() + row_ptr[r + 1];
        const int32_t *f = std::lower_bound(b, e2, cidx);
        if (f == e2 || *f != cidx) fail(HYEL_EINVAL, "mesh_upload: internal pattern error");
        return slot_of(r, (int32_t)(f - b));
    };
    for (int64_t r = 0; r < N; r++)
        for (int32_t j = 0; j < row_len[r]; j++) {
            int32_t cc = cols[row_ptr[r] + j];
            mirror[slot_of(r, j)] = (int32_t)find_slot(cc, (int32_t)r);
        }

    // ---- element pair -> slot contribution lists (ascending element order)
    std::vector<int32_t> slot_ptr(m.nslots + 1, 0), slot_list(16 * (size_t)E);
    std::vector<int32_t> pair_slot(16 * (size_t)E);
    for (int64_t e = 0; e < E; e++)
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                int64_t q = find_slot(tets[4 * e + a], tets[4 * e + b]);
                pair_slot[16 * e + 4 * a + b] = (int32_t)q;
                slot_ptr[q + 1]++;
            }
    for (int64_t q = 0; q < m.nslots; q++) slot_ptr[q + 1] += slot_ptr[q];
    {
        std::vector<int32_t> fill(slot_ptr.begin(), slot_ptr.end() - 1);
        for (int64_t e = 0; e < E; e++)
            for (int k = 0; k < 16; k++) slot_list[fill[pair_slot[16 * e + k]]++] = (int32_t)(e * kRecords + k);
    }

    // ---- boundary data
    std::vector<uint8_t> dir(N, 0);
    std::vector<double> dir_val(3 * (size_t)N, 0.0), trac(3 * (size_t)N, 0.0);
    if (bc) {
        for (int64_t k = 0; k < bc->n_dirichlet; k++) {
            int32_t n = bc->dir_node[k], cc = bc->dir_comp[k];
            if (n < 0 || n >= N || cc < 0 || cc > 2) fail(HYEL_EINVAL, "mesh_upload: Dirichlet entry out of range");
            dir[n] |= (uint8_t)(1u << cc);
            dir_val[3 * (int64_t)n + cc] = bc->dir_value ? bc->dir_value[k] : 0.0;
        }
        for (int64_t k = 0; k < bc->n_traction_tris; k++) {
            const int32_t *tr = bc->traction_tris + 3 * k;
            double P[3][3];
            for (int a = 0; a < 3; a++) {
                if (tr[a] < 0 || tr[a] >= N) fail(HYEL_EINVAL, "mesh_upload: traction node out of range");
                for (int I = 0; I < 3; I++) P[a][I] = X[3 * (int64_t)tr[a] + I];
            }
            double u[3], v[3];
            for (int I = 0; I < 3; I++) {
                u[I] = P[1][I] - P[0][I];
                v[I] = P[2][I] - P[0][I];
            }
            double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
            double area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
            for (int a = 0; a < 3; a++)
                for (int I = 0; I < 3; I++) trac[3 * (int64_t)tr[a] + I] += area / 3.0 * bc->p_max * bc->traction_dir[I];
        }
    }

    // ---- fibres
    std::vector<double> fib;
    if (mat->n_fibres == 2) {
        fib.resize(6 * (size_t)E);
        for (int64_t e = 0; e < E; e++)
            for (int I = 0; I < 3; I++) {
                fib[I * E + e] = mat->fibre_a1[3 * e + I];
                fib[(3 + I) * E + e] = mat->fibre_a2[3 * e + I];
            }
    }

    // ---- upload
    std::vector<int4> t4(E);
    for (int64_t e = 0; e < E; e++) t4[e] = make_int4(tets[4 * e], tets[4 * e + 1], tets[4 * e + 2], tets[4 * e + 3]);
    m.tets = upload(c, t4);
    m.geo = upload(c, geo);
    m.mat = upload(c, mat4);
    m.fib = upload(c, fib);
    m.slice_ptr = upload(c, slice_ptr);
    {
        std::vector<int32_t> col_slice(m.ncols);
        for (int32_t s2 = 0; s2 < m.nslices; s2++)
            for (int32_t b = slice_ptr[s2]; b < slice_ptr[s2 + 1]; b++) col_slice[b] = s2;
        m.col_slice = upload(c, col_slice);
    }
    m.row_len = upload(c, row_len);
    m.col = upload(c, col);
    m.diag_slot = upload(c, diag_slot);
    m.mirror = upload(c, mirror);
    m.slot_ptr = upload(c, slot_ptr);
    m.slot_list = upload(c, slot_list);
    m.node_ptr = upload(c, node_ptr);
    m.node_list = upload(c, node_list);
    m.dir = upload(c, dir);
    m.dir_val = upload(c, dir_val);
    m.trac = upload(c, trac);
    m.h_row_ptr = row_ptr;
    m.h_col = cols;
    m.h_csr_slot = csr_slot;
    m.h_hmax = std::move(hmax_all);
    m.h_X.assign(X, X + 3 * (size_t)N);
    m.c_m = mat->c_m;

    // ---- matrices, staging and scratch
    size_t ns = (size_t)m.nslots;
    DeviceMatrix &M = c.mat;
    M.A = dalloc_n<double>(c, 9 * ns);
    M.B = dalloc_n<double>(c, 3 * ns);
    M.C = dalloc_n<double>(c, 3 * ns);
    M.D = dalloc_n<double>(c, ns);
    M.As = dalloc_n<double>(c, 9 * ns);
    M.Bs = dalloc_n<double>(c, 3 * ns);
    M.Cs = dalloc_n<double>(c, 3 * ns);
    M.Ds = dalloc_n<double>(c, ns);
    M.Af = dalloc_n<float>(c, 9 * ns);
    M.Bf = dalloc_n<float>(c, 3 * ns);
    M.Cf = dalloc_n<float>(c, 3 * ns);
    M.Df = dalloc_n<float>(c, ns);
    M.Ah8 = dalloc_n<uint4>(c, ns);
    M.Ah1 = dalloc_n<uint16_t>(c, ns);
    M.Ahs = dalloc_n<float>(c, ns);
    M.Ams = dalloc_n<double>(c, 9 * ns);
    M.Amf = dalloc_n<float>(c, 9 * ns);
    M.Amh8 = dalloc_n<uint4>(c, ns);
    M.Amh1 = dalloc_n<uint16_t>(c, ns);
    M.Amhs = dalloc_n<float>(c, ns);
    M.w = dalloc_n<double>(c, 4 * (size_t)N);
    M.jac64 = dalloc_n<double>(c, 9 * (size_t)N);
    M.rdiag64 = dalloc_n<double>(c, 3 * (size_t)N);
    M.jac32 = dalloc_n<float>(c, 9 * (size_t)N);
    M.shat64 = dalloc_n<double>(c, (size_t)N);
    M.shat32 = dalloc_n<float>(c, (size_t)N);
    // zero the padding once: padded slots are never written by the gather
    HYEL_CK(cudaMemsetAsync(M.A, 0, 9 * ns * sizeof(double), c.stream));
    HYEL_CK(cudaMemsetAsync(M.B, 0, 3 * ns * sizeof(double), c.stream));
    HYEL_CK(cudaMemsetAsync(M.C, 0, 3 * ns * sizeof(double), c.stream));
    HYEL_CK(cudaMemsetAsync(M.D, 0, ns * sizeof(double), c.stream));
    M.At = dalloc_n<double>(c, 9 * ns);
    M.Bt = dalloc_n<double>(c, 3 * ns);
    M.Ct = dalloc_n<double>(c, 3 * ns);
    M.Dt = dalloc_n<double>(c, ns);
    HYEL_CK(cudaMemsetAsync(M.At, 0, 9 * ns * sizeof(double), c.stream));
    HYEL_CK(cudaMemsetAsync(M.Bt, 0, 3 * ns * sizeof(double), c.stream));
    HYEL_CK(cudaMemsetAsync(M.Ct, 0, 3 * ns * sizeof(double), c.stream));
    HYEL_CK(cudaMemsetAsync(M.Dt, 0, ns * sizeof(double), c.stream));
    size_t nblk32 = ((size_t)E + 31) / 32;
    c.stage = dalloc_n<double>(c, nblk32 * 32 * kRecords * kRecordDoubles);
    c.vec = dalloc_n<double>(c, 56 * (size_t)N);  // Newton states, stage values, rhs, increment
    c.red = dalloc_n<double>(c, 1 << 16);
    c.counter = dalloc_n<unsigned>(c, 64);
    c.err = dalloc_n<unsigned>(c, 4);
    HYEL_CK(cudaMemsetAsync(c.counter, 0, 64 * sizeof(unsigned), c.stream));
    HYEL_CK(cudaMemsetAsync(c.err, 0, 4 * sizeof(unsigned), c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
}

// New moduli on the uploaded mesh (mu, kappa, k1, k2, global or per element):
// material arrays and tau_M = c_m h / (c rho0) are recomputed; geometry, model
// choice, rho0, c_m, body force and fibre directions stay as uploaded.
void update_material(Ctx &c, const hyel_material *mat) {
    DeviceMesh &m = c.mesh;
    if (m.N == 0) fail(HYEL_ESTATE, "update_material: no mesh uploaded");
    if (!mat) fail(HYEL_EINVAL, "update_material: null material");
    if (mat->vol_model != m.vol_model || mat->n_fibres != m.n_fibres)
        fail(HYEL_EINVAL, "update_material: model or fibre count differs from the uploaded material");
    const int64_t E = m.E;
    std::vector<double> mat4(4 * (size_t)E), tau((size_t)E);
    for (int64_t e = 0; e < E; e++) {
        const double mu = mat->mu_e ? mat->mu_e[e] : mat->mu;
        const double kappa = mat->kappa_e ? mat->kappa_e[e] : mat->kappa;
        const double k1 = mat->k1_e ? mat->k1_e[e] : mat->k1;
        const double k2 = mat->k2_e ? mat->k2_e[e] : mat->k2;
        if (!(mu > 0)) fail(HYEL_EINVAL, "update_material: mu must be > 0");
        if (m.vol_model == HYEL_VOL_GIBBS && !(kappa > 0)) fail(HYEL_EINVAL, "update_material: kappa must be > 0");
        const double cw = m.vol_model == HYEL_VOL_GIBBS ? std::sqrt((kappa + 4.0 * mu / 3.0) / m.rho0)
                                                         : std::sqrt(mu / m.rho0);
        tau[e] = m.c_m * m.h_hmax[e] / (cw * m.rho0);
        mat4[0 * E + e] = mu;
        mat4[1 * E + e] = kappa;
        mat4[2 * E + e] = k1;
        mat4[3 * E + e] = k2;
    }
    HYEL_CK(cudaMemcpyAsync(m.mat, mat4.data(), mat4.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    HYEL_CK(cudaMemcpyAsync(m.geo + 13 * E, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    c.mat.assembled = false;
}

void mesh_upload(Ctx &c, int64_t N, const double *X, int64_t E, const int32_t *tets, const hyel_bc *bc,
                 const hyel_material *mat) {
    try {
        mesh_upload_impl(c, N, X, E, tets, bc, mat);
    } catch (...) {
        // leave the context empty (no mesh) rather than half-built
        free_workspace(c);
        amg_free(c);
        shat_free(c);
        acheb_free(c);
        dfree_all(c);
        c.mesh = DeviceMesh();
        c.mat = DeviceMatrix();
        c.stage = c.vec = c.red = nullptr;
        c.counter = c.err = nullptr;
        throw;
    }
}

}  // namespace hyel
