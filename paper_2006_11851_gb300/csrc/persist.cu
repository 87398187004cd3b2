// persist.cu -- pts_index_save / pts_index_load: an exemplar index written to a file and read
// back.  The index build is run once per exemplar and window width (section 2.2's PCA, whose
// eigen-solver dominates it), and so is the training of the learned proposal; a saved index
// skips both.
//
// File layout (host byte order, marked by a byte-order word; every field fixed-width):
//   header   "PTSINDEX", u32 version, u32 byte-order mark 0x01020304, then the scalars below
//   sections one per table, in a fixed order: u32 tag, u32 element size, u64 element count, data
// The sizes of every section follow from the header's scalars by the same formulas the build
// uses; a file whose sections disagree with them, or whose length is not exactly the sum, is
// rejected before anything is allocated on the device.
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <string>
#include <vector>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr char kMagic[8] = {'P', 'T', 'S', 'I', 'N', 'D', 'E', 'X'};
constexpr uint32_t kVersion = 2;  // 2: the channel count joined the header
constexpr uint32_t kByteOrder = 0x01020304u;
constexpr int kTreeBranch = 4;  // k of the k-means tree (section 2.2)

constexpr uint32_t tag(const char (&s)[5]) {
    return (uint32_t)s[0] | ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16) | ((uint32_t)s[3] << 24);
}

// The scalars of an index, as written.
struct Header {
    int32_t He = 0, We = 0, w = 0, D = 0, N = 0, d = 0, da = 0, d_fast = 0, da_fast = 0;
    int32_t ny = 0, nx = 0, ntiles = 0, ktc = 0, kf8 = 0, eig_iters = 0, tc_parts = 0;
    float unorm2_max = 0.0f;
    double var_retained = 0.0, eig_top = 0.0;
    int32_t prop_ready = 0, prop_C = 0;
    float prop_factor = 0.0f;
    int32_t tree_ready = 0, tree_internal = 0, tree_leaves = 0, tree_depth = 0;
    int32_t C = 3;  // channels per pixel (3 RGB, 4 RGBS)
};

// One section: its tag, element size and count as the header implies them.
struct Section {
    uint32_t tag;
    uint32_t elem;
    uint64_t count;
};

// Every section a header implies, in file order.
std::vector<Section> sections_of(const Header &h) {
    const uint64_t tcr = (uint64_t)tc_tiles(h.N) * tc_tile_rows();
    std::vector<Section> s = {
        {tag("EXEM"), 4, (uint64_t)h.He * h.We * h.C},
        {tag("EXE4"), 16, (uint64_t)h.He * h.We},
        {tag("MEAN"), 4, (uint64_t)h.D},
        {tag("BASI"), 4, (uint64_t)kMaxDPca * h.D},
        {tag("BAST"), 4, (uint64_t)h.D * kMaxDPca},
        {tag("EIGV"), 8, (uint64_t)kMaxDPca},
        {tag("ETIL"), 4, (uint64_t)h.ntiles * h.da * kBN},
        {tag("EROW"), 4, (uint64_t)h.N * h.da},
        {tag("ENRM"), 4, (uint64_t)h.ntiles * kBN},
        {tag("EFUL"), 4, (uint64_t)h.ntiles * padded_dim(h.D) * kBN},
        {tag("EFST"), 4, (uint64_t)h.ntiles * h.da_fast * kBN},
        {tag("ETCH"), 2, tcr * h.ktc},
        {tag("ETC8"), 1, tcr * h.kf8},
        {tag("F8SC"), 4, (uint64_t)h.d_fast + 1},
        {tag("UMAX"), 4, 1},
    };
    if (h.prop_ready) {
        const uint64_t C = (uint64_t)h.prop_C;
        s.push_back({tag("PCEN"), 4, C * h.d});
        s.push_back({tag("PASG"), 4, (uint64_t)h.N});
        s.push_back({tag("PCNT"), 4, C});
        s.push_back({tag("POFF"), 4, C + 1});
        s.push_back({tag("PMEM"), 4, (uint64_t)h.N});
        s.push_back({tag("PMED"), 4, C});
        s.push_back({tag("PETC"), 2, tcr * h.ktc});
        s.push_back({tag("PMLP"), 4, (uint64_t)mlp_param_count(h.prop_C)});
    }
    if (h.tree_ready) {
        s.push_back({tag("TCEN"), 4, (uint64_t)h.tree_internal * kTreeBranch * h.d});
        s.push_back({tag("TCHI"), 4, (uint64_t)h.tree_internal * kTreeBranch});
        s.push_back({tag("TLBG"), 4, (uint64_t)h.tree_leaves});
        s.push_back({tag("TLEN"), 4, (uint64_t)h.tree_leaves});
        s.push_back({tag("TPRM"), 4, (uint64_t)h.N});
    }
    return s;
}

// Field-by-field (de)serialisation of the header.
template <typename F>
void header_fields(Header &h, F &&f) {
    f(h.He), f(h.We), f(h.w), f(h.D), f(h.N), f(h.d), f(h.da), f(h.d_fast), f(h.da_fast);
    f(h.ny), f(h.nx), f(h.ntiles), f(h.ktc), f(h.kf8), f(h.eig_iters), f(h.tc_parts);
    f(h.unorm2_max), f(h.var_retained), f(h.eig_top);
    f(h.prop_ready), f(h.prop_C), f(h.prop_factor);
    f(h.tree_ready), f(h.tree_internal), f(h.tree_leaves), f(h.tree_depth);
    f(h.C);
}

// The header is consistent with an index the build could have made.
pts_status check_header(const Header &h) {
    auto bad = [](const char *what) { return set_error(PTS_ERR_INVALID_ARG, std::string("index file header: ") + what); };
    if (h.w < 1 || h.He < h.w || h.We < h.w || h.He > (1 << 16) || h.We > (1 << 16)) return bad("bad image or window size");
    if (h.C != 3 && h.C != 4) return bad("channels must be 3 or 4");
    if (h.D != h.C * h.w * h.w || h.ny != h.He - h.w + 1 || h.nx != h.We - h.w + 1) return bad("inconsistent window grid");
    const long N = (long)h.ny * h.nx;
    if (N < 2 || N > (1L << 30) || h.N != N) return bad("inconsistent window count");
    if (h.d < 1 || h.d > kMaxD || h.da != ((h.d + 1 + 3) & ~3)) return bad("bad PCA dimensions");
    if (h.d_fast < 1 || h.d_fast > kMaxDFast || h.da_fast != ((h.d_fast + 1 + 3) & ~3))
        return bad("bad tensor-core dimensions");
    if (h.ntiles != ceil_div(h.N, kBN) || h.ktc != tc_padded_k(h.d_fast) || h.kf8 != tc_padded_k8(h.d_fast))
        return bad("inconsistent tile sizes");
    if (h.tc_parts < 0 || h.eig_iters < 0) return bad("bad search settings");
    if ((h.prop_ready != 0 && h.prop_ready != 1) || (h.tree_ready != 0 && h.tree_ready != 1))
        return bad("bad proposal or tree flag");
    if (h.prop_ready && (h.prop_C < 4 || h.prop_C > 1024 || h.prop_C > h.N || !(h.prop_factor > 0.0f)))
        return bad("bad proposal sizes");
    if (h.tree_ready && (h.tree_internal < 1 || h.tree_internal > h.N || h.tree_leaves < 1 ||
                         h.tree_leaves > h.N || h.tree_depth < 0 || h.tree_depth > h.N))
        return bad("bad tree sizes");
    return PTS_OK;
}

// The integer tables the kernels index with (cluster lists, the tree's links and leaf ranges)
// are checked on the host before anything reaches the device, so a damaged file cannot make a
// kernel read or write outside its buffers.
pts_status check_tables(const Header &h, const std::vector<Section> &secs,
                        const std::vector<std::vector<unsigned char>> &data) {
    auto bad = [](const char *what) { return set_error(PTS_ERR_INVALID_ARG, std::string("index file table: ") + what); };
    auto table = [&](const char (&t)[5]) -> const int32_t * {
        for (size_t i = 0; i < secs.size(); ++i)
            if (secs[i].tag == tag(t)) return reinterpret_cast<const int32_t *>(data[i].data());
        return nullptr;
    };
    const long N = h.N;
    auto is_permutation = [&](const int32_t *p) {
        std::vector<unsigned char> seen((size_t)N, 0);
        for (long i = 0; i < N; ++i) {
            if (p[i] < 0 || p[i] >= N || seen[(size_t)p[i]]) return false;
            seen[(size_t)p[i]] = 1;
        }
        return true;
    };
    if (h.prop_ready) {
        const int C = h.prop_C;
        const int32_t *assign = table("PASG"), *cnt = table("PCNT"), *off = table("POFF"), *mem = table("PMEM");
        if (!assign || !cnt || !off || !mem) return bad("proposal tables missing");
        if (off[0] != 0 || off[C] != N) return bad("cluster offsets do not run from 0 to N");
        for (int c = 0; c < C; ++c)
            if (off[c + 1] < off[c] || cnt[c] != off[c + 1] - off[c]) return bad("cluster offsets or sizes");
        for (long i = 0; i < N; ++i)
            if (assign[i] < 0 || assign[i] >= C) return bad("a window's cluster is out of range");
        if (!is_permutation(mem)) return bad("cluster members are not a permutation of the windows");
        for (int c = 0; c < C; ++c)
            for (int i = off[c]; i < off[c + 1]; ++i)
                if (assign[mem[i]] != c) return bad("a cluster lists a window of another cluster");
    }
    if (h.tree_ready) {
        const int32_t *child = table("TCHI"), *lb = table("TLBG"), *le = table("TLEN"), *perm = table("TPRM");
        if (!child || !lb || !le || !perm) return bad("tree tables missing");
        for (long node = 0; node < h.tree_internal; ++node)
            for (int k = 0; k < kTreeBranch; ++k) {
                const int32_t c = child[node * kTreeBranch + k];
                // internal children come after their parent (nodes are numbered level by level),
                // which also rules out cycles
                const bool internal = c >= 0 && c > node && c < h.tree_internal;
                const bool leaf = c <= -2 && (long)(-(long)c - 2) < h.tree_leaves;
                if (c != -1 && !internal && !leaf) return bad("a tree child reference is out of range");
            }
        for (long l = 0; l < h.tree_leaves; ++l)
            if (lb[l] < 0 || lb[l] > le[l] || le[l] > N) return bad("a tree leaf range is out of range");
        if (!is_permutation(perm)) return bad("the tree's window order is not a permutation");
    }
    return PTS_OK;
}

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

pts_status write_all(FILE *f, const void *p, size_t n, const char *path) {
    if (n && fwrite(p, 1, n, f) != n) return set_error(PTS_ERR_INVALID_ARG, std::string("pts_index_save: write failed: ") + path);
    return PTS_OK;
}

pts_status read_all(FILE *f, void *p, size_t n) {
    if (n && fread(p, 1, n, f) != n) return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: file ends early");
    return PTS_OK;
}

// Device pointer of each section of an index, in file order (the tables must exist).
std::vector<void *> device_tables(pts_index idx, const Header &h) {
    std::vector<void *> p = {idx->exemplar.ptr, idx->exemplar4.ptr, idx->mu.ptr,     idx->basis.ptr, idx->basisT.ptr,
                             idx->eig.ptr,      idx->et.ptr,        idx->et_rows.ptr, idx->enorm.ptr, idx->efull.ptr,
                             idx->et_fast.ptr,  idx->etc.ptr,       idx->etc8.ptr,   idx->f8scale.ptr, idx->umax.ptr};
    if (h.prop_ready) {
        ProposalState &pr = idx->prop;
        for (void *q : {(void *)pr.centroids.ptr, (void *)pr.assign.ptr, (void *)pr.counts.ptr, (void *)pr.off.ptr,
                        (void *)pr.members.ptr, (void *)pr.median.ptr, (void *)pr.etc_ivf.ptr, (void *)pr.mlp.params.ptr})
            p.push_back(q);
    }
    if (h.tree_ready) {
        KmTree &tr = idx->tree;
        for (void *q : {(void *)tr.cent.ptr, (void *)tr.child.ptr, (void *)tr.leaf_begin.ptr, (void *)tr.leaf_end.ptr,
                        (void *)tr.perm.ptr})
            p.push_back(q);
    }
    return p;
}

}  // namespace
}  // namespace pts

using namespace pts;

extern "C" {

pts_status pts_index_save(pts_index idx, const char *path) {
    if (!idx || !path || !*path) return set_error(PTS_ERR_INVALID_ARG, "pts_index_save: null index or path");
    Header h;
    h.He = idx->He, h.We = idx->We, h.w = idx->w, h.D = idx->D, h.N = idx->N, h.d = idx->d, h.da = idx->da;
    h.d_fast = idx->d_fast, h.da_fast = idx->da_fast, h.ny = idx->ny, h.nx = idx->nx, h.ntiles = idx->ntiles;
    h.ktc = idx->ktc, h.kf8 = idx->kf8, h.eig_iters = idx->eig_iters, h.tc_parts = idx->tc_parts_override;
    h.unorm2_max = idx->unorm2_max, h.var_retained = idx->var_retained, h.eig_top = idx->eig_top;
    h.prop_ready = idx->prop.ready ? 1 : 0, h.prop_C = idx->prop.ready ? idx->prop.C : 0;
    h.prop_factor = idx->prop.ready ? idx->prop.factor : 0.0f;
    h.tree_ready = idx->tree.ready ? 1 : 0;
    h.tree_internal = idx->tree.ready ? idx->tree.n_internal : 0;
    h.tree_leaves = idx->tree.ready ? idx->tree.n_leaves : 0;
    h.tree_depth = idx->tree.ready ? idx->tree.depth : 0;
    h.C = idx->C;
    PTS_TRY(check_header(h));
    const std::vector<Section> secs = sections_of(h);
    const std::vector<void *> dev = device_tables(idx, h);
    PTS_CUDA_TRY(cudaSetDevice(idx->device));
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    // write to a temporary name, then rename, so a failed save never leaves a partial file
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    pts_status s = PTS_OK;
    {
        File f;
        f.f = fopen(tmp.c_str(), "wb");
        if (!f.f) return set_error(PTS_ERR_INVALID_ARG, std::string("pts_index_save: cannot open ") + tmp);
        s = write_all(f.f, kMagic, sizeof(kMagic), path);
        if (s == PTS_OK) s = write_all(f.f, &kVersion, 4, path);
        if (s == PTS_OK) s = write_all(f.f, &kByteOrder, 4, path);
        header_fields(h, [&](auto &v) {
            if (s == PTS_OK) s = write_all(f.f, &v, sizeof(v), path);
        });
        std::vector<unsigned char> host;
        for (size_t i = 0; s == PTS_OK && i < secs.size(); ++i) {
            const Section &c = secs[i];
            const size_t bytes = (size_t)c.elem * c.count;
            host.resize(bytes);
            cudaError_t e = cudaMemcpy(host.data(), dev[i], bytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                s = cuda_error(e, "pts_index_save: read table");
                break;
            }
            s = write_all(f.f, &c.tag, 4, path);
            if (s == PTS_OK) s = write_all(f.f, &c.elem, 4, path);
            if (s == PTS_OK) s = write_all(f.f, &c.count, 8, path);
            if (s == PTS_OK) s = write_all(f.f, host.data(), bytes, path);
        }
        if (s == PTS_OK && fflush(f.f) != 0) s = set_error(PTS_ERR_INVALID_ARG, "pts_index_save: flush failed");
    }
    if (s == PTS_OK && rename(tmp.c_str(), path) != 0)
        s = set_error(PTS_ERR_INVALID_ARG, std::string("pts_index_save: cannot rename to ") + path);
    if (s != PTS_OK) unlink(tmp.c_str());
    return s;
}

pts_status pts_index_load(const char *path, pts_index *out) {
    if (!out || !path || !*path) return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: null path or output");
    *out = nullptr;
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return set_error(PTS_ERR_INVALID_ARG, std::string("pts_index_load: cannot open ") + path);
    char magic[8];
    uint32_t version = 0, order = 0;
    PTS_TRY(read_all(f.f, magic, 8));
    if (memcmp(magic, kMagic, 8) != 0) return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: not an index file");
    PTS_TRY(read_all(f.f, &version, 4));
    PTS_TRY(read_all(f.f, &order, 4));
    if (order != kByteOrder) return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: written with another byte order");
    if (version != kVersion) return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: unknown file version");
    Header h;
    pts_status s = PTS_OK;
    header_fields(h, [&](auto &v) {
        if (s == PTS_OK) s = read_all(f.f, &v, sizeof(v));
    });
    PTS_TRY(s);
    PTS_TRY(check_header(h));
    const std::vector<Section> secs = sections_of(h);
    // the whole length is checked before any device work
    const long pos = ftell(f.f);
    uint64_t expect = (uint64_t)pos;
    for (const Section &c : secs) expect += 16 + (uint64_t)c.elem * c.count;
    struct stat stt;
    if (fstat(fileno(f.f), &stt) != 0 || (uint64_t)stt.st_size != expect)
        return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: file length does not match its header");

    // read and check every section on the host before any device work
    std::vector<std::vector<unsigned char>> data(secs.size());
    for (size_t i = 0; i < secs.size(); ++i) {
        Section c{0, 0, 0};
        PTS_TRY(read_all(f.f, &c.tag, 4));
        PTS_TRY(read_all(f.f, &c.elem, 4));
        PTS_TRY(read_all(f.f, &c.count, 8));
        if (c.tag != secs[i].tag || c.elem != secs[i].elem || c.count != secs[i].count)
            return set_error(PTS_ERR_INVALID_ARG, "pts_index_load: a section does not match the header");
        data[i].resize((size_t)c.elem * c.count);
        PTS_TRY(read_all(f.f, data[i].data(), data[i].size()));
    }
    PTS_TRY(check_tables(h, secs, data));

    pts_index idx = new pts_index_s();
    register_index(idx);
    auto fail = [&](pts_status st) {
        pts_index_destroy(idx);
        return st;
    };
    if (cudaGetDevice(&idx->device) != cudaSuccess) {
        cudaGetLastError();
        unregister_index(idx);
        delete idx;
        return set_error(PTS_ERR_CUDA, "pts_index_load: no CUDA device");
    }
    idx->He = h.He, idx->We = h.We, idx->w = h.w, idx->D = h.D, idx->N = h.N, idx->d = h.d, idx->da = h.da;
    idx->C = h.C;
    idx->d_fast = h.d_fast, idx->da_fast = h.da_fast, idx->ny = h.ny, idx->nx = h.nx, idx->ntiles = h.ntiles;
    idx->ktc = h.ktc, idx->kf8 = h.kf8, idx->eig_iters = h.eig_iters, idx->tc_parts_override = h.tc_parts;
    idx->unorm2_max = h.unorm2_max, idx->var_retained = h.var_retained, idx->eig_top = h.eig_top;
    // allocate every table at the size the build gives it
    const uint64_t tcr = (uint64_t)tc_tiles(h.N) * tc_tile_rows();
    if ((s = idx->exemplar.ensure((size_t)h.He * h.We * h.C, "exemplar")) != PTS_OK) return fail(s);
    if ((s = idx->exemplar4.ensure((size_t)h.He * h.We, "exemplar rgba")) != PTS_OK) return fail(s);
    if ((s = idx->mu.ensure(h.D, "mean")) != PTS_OK) return fail(s);
    if ((s = idx->basis.ensure((size_t)kMaxDPca * h.D, "basis")) != PTS_OK) return fail(s);
    if ((s = idx->basisT.ensure((size_t)h.D * kMaxDPca, "transposed basis")) != PTS_OK) return fail(s);
    if ((s = idx->eig.ensure(kMaxDPca, "eigenvalues")) != PTS_OK) return fail(s);
    if ((s = idx->et.ensure((size_t)h.ntiles * h.da * kBN, "exemplar vectors")) != PTS_OK) return fail(s);
    if ((s = idx->et_rows.ensure((size_t)h.N * h.da, "window-major exemplar vectors")) != PTS_OK) return fail(s);
    if ((s = idx->enorm.ensure((size_t)h.ntiles * kBN, "exemplar norms")) != PTS_OK) return fail(s);
    if ((s = idx->efull.ensure((size_t)h.ntiles * padded_dim(h.D) * kBN, "full exemplar vectors")) != PTS_OK)
        return fail(s);
    if ((s = idx->et_fast.ensure((size_t)h.ntiles * h.da_fast * kBN, "fast exemplar vectors")) != PTS_OK)
        return fail(s);
    if ((s = idx->etc.ensure(tcr * h.ktc, "fp16 exemplar tiles")) != PTS_OK) return fail(s);
    if ((s = idx->etc8.ensure(tcr * h.kf8, "fp8 exemplar tiles")) != PTS_OK) return fail(s);
    if ((s = idx->f8scale.ensure((size_t)h.d_fast + 1, "fp8 scales")) != PTS_OK) return fail(s);
    if ((s = idx->umax.ensure(1, "norm max")) != PTS_OK) return fail(s);
    if ((s = idx->status.ensure(1, "status")) != PTS_OK) return fail(s);
    ProposalState &pr = idx->prop;
    if (h.prop_ready) {
        const size_t C = (size_t)h.prop_C;
        if ((s = pr.centroids.ensure(C * h.d, "centroids")) != PTS_OK) return fail(s);
        if ((s = pr.assign.ensure(h.N, "cluster of each window")) != PTS_OK) return fail(s);
        if ((s = pr.counts.ensure(C, "cluster sizes")) != PTS_OK) return fail(s);
        if ((s = pr.off.ensure(C + 1, "cluster offsets")) != PTS_OK) return fail(s);
        if ((s = pr.members.ensure(h.N, "cluster members")) != PTS_OK) return fail(s);
        if ((s = pr.median.ensure(C, "cluster medians")) != PTS_OK) return fail(s);
        if ((s = pr.etc_ivf.ensure(tcr * h.ktc, "cluster-ordered tiles")) != PTS_OK) return fail(s);
        // weights only: the search sizes the activation buffers it needs on first use
        if ((s = pr.mlp.ensure(h.prop_C, 0, nullptr)) != PTS_OK) return fail(s);
    }
    KmTree &tr = idx->tree;
    if (h.tree_ready) {
        if ((s = tr.cent.ensure((size_t)h.tree_internal * kTreeBranch * h.d, "tree centroids")) != PTS_OK)
            return fail(s);
        if ((s = tr.child.ensure((size_t)h.tree_internal * kTreeBranch, "tree children")) != PTS_OK) return fail(s);
        if ((s = tr.leaf_begin.ensure(h.tree_leaves, "tree leaves")) != PTS_OK) return fail(s);
        if ((s = tr.leaf_end.ensure(h.tree_leaves, "tree leaves")) != PTS_OK) return fail(s);
        if ((s = tr.perm.ensure(h.N, "tree permutation")) != PTS_OK) return fail(s);
    }
    // upload the checked sections
    const std::vector<void *> dev = device_tables(idx, h);
    for (size_t i = 0; i < secs.size(); ++i) {
        cudaError_t e = cudaMemcpy(dev[i], data[i].data(), data[i].size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_error(e, "pts_index_load: upload table"));
    }
    if (cudaMemset(idx->status.ptr, 0, sizeof(int)) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "status"));
    // the window-major copy of the fast vectors and their variance fraction follow from the tables
    if ((s = idx->et_fast_rows.ensure((size_t)h.N * h.da_fast, "window-major fast exemplar vectors")) != PTS_OK)
        return fail(s);
    launch_tiles_to_rows(idx->et_fast.ptr, h.N, h.da_fast, idx->et_fast_rows.ptr, nullptr);
    {
        const double *ev = nullptr;
        for (size_t i = 0; i < secs.size(); ++i)
            if (secs[i].tag == tag("EIGV")) ev = reinterpret_cast<const double *>(data[i].data());
        double kept_d = 0.0, kept_fast = 0.0;
        for (int j = 0; j < h.d; ++j) kept_d += ev[j];
        for (int j = 0; j < h.d_fast && j < kMaxDPca; ++j) kept_fast += ev[j];
        idx->var_fast = kept_d > 0.0 ? h.var_retained * kept_fast / kept_d : 0.0;
    }
    if (h.prop_ready) {
        // the network's BF16 weights and the inference kernel's packed copy follow from the FP32
        // weights exactly as at the end of training
        pr.C = h.prop_C;
        pr.factor = h.prop_factor;
        mlp_refresh_bf16(pr.mlp, nullptr);
        if ((s = mlp_pack_infer(pr.mlp, pr.infer, nullptr)) != PTS_OK) return fail(s);
        pr.ready = 1;
    }
    if (h.tree_ready) {
        tr.n_internal = h.tree_internal;
        tr.n_leaves = h.tree_leaves;
        tr.depth = h.tree_depth;
        tr.d = h.d;
        tr.N = h.N;
        tr.ready = 1;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(cuda_error(e, "pts_index_load"));
    *out = idx;
    return PTS_OK;
}

}  // extern "C"
