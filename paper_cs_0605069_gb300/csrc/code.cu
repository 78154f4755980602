// Code objects: validation of H, GF(2^p) tables, CSR/CSC index arrays and
// their single device allocation (Sec. 2: row i of H lists the symbols of
// check i, column j the checks of symbol j).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "gfbp_internal.cuh"

namespace gfbp {
void set_error(const std::string& msg);
}

using gfbp::set_error;

namespace {

uint32_t default_poly(int p) {
    static const uint32_t polys[9] = {0, 0x3, 0x7, 0xB, 0x13, 0x25, 0x43, 0x89, 0x11D};
    return (p >= 1 && p <= 8) ? polys[p] : 0;
}

int log2_exact(int q) {
    for (int p = 1; p <= 8; p++)
        if ((1 << p) == q) return p;
    return -1;
}

// exp/log tables of the primitive element x; false if poly is not primitive.
bool build_field(int q, int p, uint32_t poly, uint8_t* ex, uint8_t* lg) {
    if ((poly >> p) != 1u) return false;
    std::vector<int> seen(q, -1);
    uint32_t v = 1;
    for (int i = 0; i < q - 1; i++) {
        if (seen[v] != -1) return false;
        seen[v] = i;
        ex[i] = (uint8_t)v;
        lg[v] = (uint8_t)i;
        v <<= 1;
        if (v & (uint32_t)q) v ^= poly;
    }
    if (v != 1u) return false;
    for (int i = q - 1; i < 512; i++) ex[i] = ex[i % (q - 1)];
    lg[0] = 0;
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// H's index arrays and the SUS level schedule, built on the host.
struct HostCode {
    std::vector<int> rowptr, colptr, ecol, erow, cedge, cpred, lev, lpiece;
    std::vector<uint8_t> eh, cdep;
    std::vector<int4> cinfo, lrec;
    std::vector<int2> lpair, lpair_d;
    int dcmax = 0, dvmax = 0, nlevels = 0, npieces = 0;
};

// Validates the COO entries (ranges, duplicates, degree limits) and fills h;
// `who` names the caller in error messages.
gfbp_status build_host(int q, int M, int N, int64_t nnz, const int32_t* row, const int32_t* col, const int32_t* val,
                       HostCode& h, const char* who) {
    auto& rowptr = h.rowptr;
    auto& colptr = h.colptr;
    auto& ecol = h.ecol;
    auto& erow = h.erow;
    auto& cedge = h.cedge;
    auto& cpred = h.cpred;
    auto& lev = h.lev;
    auto& lpiece = h.lpiece;
    auto& eh = h.eh;
    auto& cdep = h.cdep;
    auto& cinfo = h.cinfo;
    auto& lrec = h.lrec;
    auto& lpair = h.lpair;
    auto& lpair_d = h.lpair_d;
    int& dcmax = h.dcmax;
    int& dvmax = h.dvmax;
    int& nlevels = h.nlevels;
    int& npieces = h.npieces;
    const long long E = nnz;
    std::vector<long long> order(E);
    for (long long e = 0; e < E; e++) {
        if (row[e] < 0 || row[e] >= M || col[e] < 0 || col[e] >= N || val[e] < 1 || val[e] >= q) {
            set_error(std::string(who) + ": COO entry " + std::to_string(e) + " out of range");
            return GFBP_EINVAL;
        }
        order[e] = e;
    }
    std::sort(order.begin(), order.end(), [&](long long a, long long b) {
        return row[a] != row[b] ? row[a] < row[b] : col[a] < col[b];
    });
    rowptr.assign(M + 1, 0);
    colptr.assign(N + 1, 0);
    ecol.assign(E, 0);
    erow.assign(E, 0);
    cedge.assign(E, 0);
    eh.assign(E, 0);
    for (long long k = 0; k < E; k++) {
        const long long e = order[k];
        if (k > 0 && row[order[k - 1]] == row[e] && col[order[k - 1]] == col[e]) {
            set_error(std::string(who) + ": duplicate (row, col) entry");
            return GFBP_EINVAL;
        }
        erow[k] = row[e];
        ecol[k] = col[e];
        eh[k] = (uint8_t)val[e];
        rowptr[row[e] + 1]++;
        colptr[col[e] + 1]++;
    }
    for (int i = 0; i < M; i++) rowptr[i + 1] += rowptr[i];
    for (int j = 0; j < N; j++) colptr[j + 1] += colptr[j];
    {
        std::vector<int> fill(N, 0);
        for (long long k = 0; k < E; k++) cedge[colptr[ecol[k]] + fill[ecol[k]]++] = (int)k;
    }
    dcmax = 0;
    dvmax = 0;
    for (int i = 0; i < M; i++) dcmax = std::max(dcmax, rowptr[i + 1] - rowptr[i]);
    for (int j = 0; j < N; j++) dvmax = std::max(dvmax, colptr[j + 1] - colptr[j]);
    if (dcmax > 16 || dvmax > 8) {
        set_error(std::string(who) + ": row degree must be <= 16 and column degree <= 8");
        return GFBP_EUNSUPPORTED;
    }

    // per column slot: {edge, row start, row degree | h << 8, row}; and whether
    // column j shares a check with column j-1 (SUS prefetch must then reload)
    cinfo.assign(E, make_int4(0, 0, 0, 0));
    cdep.assign(N, 0);
    // and the last earlier column that shares a check with column j (-1 if
    // none): SUS may run column j once every column up to that one is done
    cpred.assign(N, -1);
    for (int j = 0; j < N; j++) {
        for (int k = colptr[j]; k < colptr[j + 1]; k++) {
            const int e = cedge[k], i = erow[e];
            cinfo[k] = make_int4(e, rowptr[i], (rowptr[i + 1] - rowptr[i]) | ((int)eh[e] << 8), i);
            if (j > 0)
                for (int k2 = colptr[j - 1]; k2 < colptr[j]; k2++)
                    if (erow[cedge[k2]] == i) cdep[j] = 1;
            for (int e2 = rowptr[i]; e2 < rowptr[i + 1]; e2++)
                if (ecol[e2] < j) cpred[j] = std::max(cpred[j], ecol[e2]);
        }
    }

    // SUS level schedule and its pieces (whole columns of one level, at most
    // kLevelPiece (column, slot) pairs each)
    lev.assign(N, 0);
    nlevels = 0;
    for (int j = 0; j < N; j++) {
        int m = -1;
        for (int k = colptr[j]; k < colptr[j + 1]; k++) {
            const int i = erow[cedge[k]];
            for (int e2 = rowptr[i]; e2 < rowptr[i + 1]; e2++)
                if (ecol[e2] < j) m = std::max(m, lev[ecol[e2]]);
        }
        lev[j] = m + 1;
        nlevels = std::max(nlevels, lev[j] + 1);
    }
    std::vector<int> lorder(N);
    {
        std::vector<int> cnt(nlevels + 1, 0);
        for (int j = 0; j < N; j++) cnt[lev[j] + 1]++;
        for (int l = 0; l < nlevels; l++) cnt[l + 1] += cnt[l];
        for (int j = 0; j < N; j++) lorder[cnt[lev[j]]++] = j;
    }
    lpair.clear();
    lpiece.assign(1, 0);
    lpair.reserve(E + N);
    {
        int cur = -1, in_piece = 0;
        for (int j : lorder) {
            const int d = colptr[j + 1] - colptr[j];
            // a column without checks gets one pair (j, 0): only its posterior
            const int np = d > 0 ? d : 1;
            if (lev[j] != cur || in_piece + np > gfbp::kLevelPiece) {
                if (in_piece) lpiece.push_back((int)lpair.size());
                in_piece = 0;
                cur = lev[j];
            }
            for (int k = 0; k < np; k++) lpair.push_back(make_int2(j, k));
            in_piece += np;
        }
        if (in_piece) lpiece.push_back((int)lpair.size());
    }
    npieces = (int)lpiece.size() - 1;
    // The same pairs for the q <= 16 level kernel, reordered inside each piece
    // by the work the running partial convolutions give them (a convolution
    // in both steps for a check position 1..d_c-2, none otherwise) so that a
    // warp's threads take the same branch; .y = slot | (index of the pair in
    // the column-ordered piece) << 8, which keeps a column's rows adjacent.
    lpair_d.assign(lpair.size(), make_int2(0, 0));
    for (int pc = 0; pc < npieces; pc++) {
        const int s = lpiece[pc], e = lpiece[pc + 1];
        int o = s;
        for (int cls = 0; cls < 3; cls++)
            for (int x = s; x < e; x++) {
                const int j = lpair[x].x, k = lpair[x].y;
                int c = 2;   // last position of its check, a check of degree 1, or no check
                if (colptr[j + 1] > colptr[j]) {
                    const int4 in = cinfo[colptr[j] + k];
                    const int t = in.x - in.y, dc = in.z & 255;
                    if (dc >= 2 && t == 0) c = 1;
                    else if (t >= 1 && t <= dc - 2) c = 0;
                }
                if (c == cls) lpair_d[o++] = make_int2(j, k | ((x - s) << 8));
            }
    }
    // per entry of lpair_d: the slot's cinfo (zeros for a column without
    // checks) and {column, slot | row index << 8, column degree, 0}
    lrec.assign(2 * lpair_d.size(), make_int4(0, 0, 0, 0));
    for (size_t x = 0; x < lpair_d.size(); x++) {
        const int j = lpair_d[x].x, k = lpair_d[x].y & 255;
        const int d = colptr[j + 1] - colptr[j];
        lrec[2 * x] = d > 0 ? cinfo[colptr[j] + k] : make_int4(0, 0, 0, 0);
        lrec[2 * x + 1] = make_int4(j, lpair_d[x].y, d, 0);
    }

    return GFBP_OK;
}


}  // namespace

extern "C" gfbp_status gfbp_code_create(int32_t q, int32_t M, int32_t N, int64_t nnz, const int32_t* row,
                                        const int32_t* col, const int32_t* val, uint32_t prim_poly,
                                        gfbp_code** out) {
    if (!out) { set_error("gfbp_code_create: out is NULL"); return GFBP_EINVAL; }
    *out = nullptr;
    const int p = log2_exact(q);
    if (p < 0) { set_error("gfbp_code_create: q must be 2^p with 1 <= p <= 8"); return GFBP_EINVAL; }
    if (M < 0 || N < 1 || nnz < 0 || nnz > (int64_t)1 << 31) {
        set_error("gfbp_code_create: need M >= 0, N >= 1, 0 <= nnz < 2^31");
        return GFBP_EINVAL;
    }
    if (nnz > 0 && (!row || !col || !val)) { set_error("gfbp_code_create: NULL COO array"); return GFBP_EINVAL; }
    const uint32_t poly = prim_poly ? prim_poly : default_poly(p);
    uint8_t ex[512] = {0}, lg[256] = {0};
    if (!build_field(q, p, poly, ex, lg)) {
        set_error("gfbp_code_create: field polynomial is not primitive of degree log2(q)");
        return GFBP_EINVAL;
    }
    HostCode h;
    {
        const gfbp_status st = build_host(q, M, N, nnz, row, col, val, h, "gfbp_code_create");
        if (st != GFBP_OK) return st;
    }
    const long long E = nnz;
    const std::vector<int>&rowptr = h.rowptr, &colptr = h.colptr, &ecol = h.ecol, &erow = h.erow, &cedge = h.cedge,
                    &cpred = h.cpred, &lpiece = h.lpiece;
    const std::vector<uint8_t>&eh = h.eh, &cdep = h.cdep;
    const std::vector<int4>&cinfo = h.cinfo, &lrec = h.lrec;
    const std::vector<int2>&lpair = h.lpair, &lpair_d = h.lpair_d;
    const int dcmax = h.dcmax, dvmax = h.dvmax, nlevels = h.nlevels, npieces = h.npieces;
    // one device allocation: rowptr | colptr | ecol | erow | cedge | eh | gexp | glog | cinfo | cdep | cpred |
    // lpair | lpiece | lpair_d | lrec
    constexpr int NA = 15;
    size_t off[NA], total = 0;
    const size_t sz[] = {sizeof(int) * (size_t)(M + 1), sizeof(int) * (size_t)(N + 1), sizeof(int) * (size_t)E,
                           sizeof(int) * (size_t)E,       sizeof(int) * (size_t)E,       (size_t)E,
                           512,                           256,                           sizeof(int4) * (size_t)E,
                           (size_t)N,                     sizeof(int) * (size_t)N,       sizeof(int2) * lpair.size(),
                           sizeof(int) * lpiece.size(),   sizeof(int2) * lpair_d.size(),
                           sizeof(int4) * lrec.size()};
    static_assert(sizeof(sz) / sizeof(sz[0]) == NA, "one size per array");
    for (int k = 0; k < NA; k++) { off[k] = total; total += align256(sz[k] ? sz[k] : 1); }
    std::vector<uint8_t> host(total, 0);
    std::memcpy(host.data() + off[0], rowptr.data(), sz[0]);
    std::memcpy(host.data() + off[1], colptr.data(), sz[1]);
    if (E) {
        std::memcpy(host.data() + off[2], ecol.data(), sz[2]);
        std::memcpy(host.data() + off[3], erow.data(), sz[3]);
        std::memcpy(host.data() + off[4], cedge.data(), sz[4]);
        std::memcpy(host.data() + off[5], eh.data(), sz[5]);
        std::memcpy(host.data() + off[8], cinfo.data(), sz[8]);
    }
    std::memcpy(host.data() + off[6], ex, 512);
    std::memcpy(host.data() + off[7], lg, 256);
    std::memcpy(host.data() + off[9], cdep.data(), sz[9]);
    std::memcpy(host.data() + off[10], cpred.data(), sz[10]);
    if (!lpair.empty()) std::memcpy(host.data() + off[11], lpair.data(), sz[11]);
    std::memcpy(host.data() + off[12], lpiece.data(), sz[12]);
    if (!lpair_d.empty()) std::memcpy(host.data() + off[13], lpair_d.data(), sz[13]);
    if (!lrec.empty()) std::memcpy(host.data() + off[14], lrec.data(), sz[14]);

    gfbp_code* c = new (std::nothrow) gfbp_code();
    if (!c) { set_error("gfbp_code_create: out of host memory"); return GFBP_ENOMEM; }
    cudaError_t err = cudaGetDevice(&c->device);
    if (err == cudaSuccess) err = cudaMalloc(&c->dmem, total);
    if (err != cudaSuccess) {
        set_error(std::string("gfbp_code_create: ") + cudaGetErrorString(err));
        delete c;
        return err == cudaErrorMemoryAllocation ? GFBP_ENOMEM : GFBP_ECUDA;
    }
    err = cudaMemcpy(c->dmem, host.data(), total, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        set_error(std::string("gfbp_code_create: ") + cudaGetErrorString(err));
        cudaFree(c->dmem);
        delete c;
        return GFBP_ECUDA;
    }
    uint8_t* base = static_cast<uint8_t*>(c->dmem);
    gfbp::CodeDev& d = c->dev;
    d.q = q; d.p = p; d.M = M; d.N = N; d.E = E; d.dcmax = dcmax; d.dvmax = dvmax;
    d.rowptr = reinterpret_cast<const int*>(base + off[0]);
    d.colptr = reinterpret_cast<const int*>(base + off[1]);
    d.ecol = reinterpret_cast<const int*>(base + off[2]);
    d.erow = reinterpret_cast<const int*>(base + off[3]);
    d.cedge = reinterpret_cast<const int*>(base + off[4]);
    d.eh = base + off[5];
    d.gexp = base + off[6];
    d.glog = base + off[7];
    d.cinfo = reinterpret_cast<const int4*>(base + off[8]);
    d.cdep = base + off[9];
    d.cpred = reinterpret_cast<const int*>(base + off[10]);
    d.nlevels = nlevels;
    d.npieces = npieces;
    d.lpair = reinterpret_cast<const int2*>(base + off[11]);
    d.lpiece = reinterpret_cast<const int*>(base + off[12]);
    d.lpair_d = reinterpret_cast<const int2*>(base + off[13]);
    d.lrec = reinterpret_cast<const int4*>(base + off[14]);
    c->poly = poly;
    *out = c;
    return GFBP_OK;
}

extern "C" void gfbp_code_destroy(gfbp_code* code) {
    if (!code) return;
    cudaFree(code->dmem);
    delete code;
}

extern "C" gfbp_status gfbp_code_info(const gfbp_code* code, int32_t* q, int32_t* M, int32_t* N, int64_t* E,
                                      int32_t* max_row_degree, int32_t* max_col_degree) {
    if (!code) { set_error("gfbp_code_info: NULL code"); return GFBP_EINVAL; }
    if (q) *q = code->dev.q;
    if (M) *M = code->dev.M;
    if (N) *N = code->dev.N;
    if (E) *E = code->dev.E;
    if (max_row_degree) *max_row_degree = code->dev.dcmax;
    if (max_col_degree) *max_col_degree = code->dev.dvmax;
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_level_schedule(int32_t q, int32_t M, int32_t N, int64_t nnz, const int32_t* row,
                                           const int32_t* col, const int32_t* val, int32_t* level,
                                           int32_t* n_levels, int32_t* piece_ptr, int32_t* n_pieces,
                                           int32_t* pair_col, int32_t* pair_slot, int32_t* pair_row,
                                           int32_t* n_pairs) {
    if (log2_exact(q) < 0) { set_error("gfbp_level_schedule: q must be 2^p with 1 <= p <= 8"); return GFBP_EINVAL; }
    if (M < 0 || N < 1 || nnz < 0 || nnz > (int64_t)1 << 31) {
        set_error("gfbp_level_schedule: need M >= 0, N >= 1, 0 <= nnz < 2^31");
        return GFBP_EINVAL;
    }
    if (nnz > 0 && (!row || !col || !val)) { set_error("gfbp_level_schedule: NULL COO array"); return GFBP_EINVAL; }
    if (!level || !n_levels || !piece_ptr || !n_pieces || !pair_col || !pair_slot || !pair_row || !n_pairs) {
        set_error("gfbp_level_schedule: NULL output");
        return GFBP_EINVAL;
    }
    HostCode h;
    const gfbp_status st = build_host(q, M, N, nnz, row, col, val, h, "gfbp_level_schedule");
    if (st != GFBP_OK) return st;
    for (int j = 0; j < N; j++) level[j] = h.lev[j];
    *n_levels = h.nlevels;
    for (int pc = 0; pc <= h.npieces; pc++) piece_ptr[pc] = h.lpiece[pc];
    *n_pieces = h.npieces;
    for (size_t x = 0; x < h.lpair_d.size(); x++) {
        pair_col[x] = h.lpair_d[x].x;
        pair_slot[x] = h.lpair_d[x].y & 255;
        pair_row[x] = h.lpair_d[x].y >> 8;
    }
    *n_pairs = (int32_t)h.lpair_d.size();
    return GFBP_OK;
}
