// Batches of frames of several codes — uneven q and N — decoded by ONE
// persistent launch (per schedule) over a device frame table, with no host
// synchronisation or allocation after gfbp_batch_create, so that a run can be
// captured in a CUDA graph and replayed.  Each item carries the kernel variant
// that decodes its frames, chosen by the autotuner (gfbp_autotune) or by
// default rules.  SUS variants come in two families: the level schedules (a
// CTA per frame: a thread per (column, check) pair for the probability route,
// a lane group per pair for the transform route) and the column walkers (a
// warp per frame: team or group kernels); a run launches one persistent
// kernel per family present, each over the frame table, skipping the other
// family's frames.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "pus_frame.cuh"
#include "sus_group.cuh"
#include "sus_level.cuh"
#include "sus_level_tc.cuh"
#include "sus_level_tr.cuh"
#include "sus_team.cuh"

namespace gfbp {
void set_error(const std::string& msg);
cudaError_t batch_prepare_item(DecodeArgs& A, void* ws, const gfbp_code* code, int32_t F, const float* obs,
                               gfbp_channel ch, gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter,
                               uint8_t* x_hat, int32_t* iters, uint8_t* conv, const gfbp_options* opt,
                               int method, size_t* ws_bytes, cudaStream_t stream);
cudaError_t launch_fill_prior(const DecodeArgs& A, cudaStream_t s);
}  // namespace gfbp

namespace gfbp {
namespace {

constexpr int kMaxItems = 65536;
constexpr int kMixedThreads = 128;  // SUS: 4 warps, one frame per warp

// Kernel variants a batch item can use (codes with row degree <= 6 and column
// degree <= 3; other codes are decoded by gfbp_decode).
enum Variant : int {
    kTeam4 = 0, kTeam8, kTeam16,                              // SUS team, probability route
    kGroup2D, kGroup4D, kGroup8D, kGroup16D,                  // SUS group, probability route
    kGroup32T, kGroup64T, kGroup128T, kGroup256T,             // SUS group, transform route
    kLevel2D, kLevel4D, kLevel8D, kLevel16D,                  // SUS levels, probability route (CTA family)
    kLevel32T, kLevel64T, kLevel128T, kLevel256T,             // SUS levels, transform route (CTA family)
    kLevel16X, kLevel32X, kLevel64X, kLevel128X, kLevel256X,  // SUS levels, tensor-core route (CTA family)
    kLevel32D, kLevel64D, kLevel128D, kLevel256D,             // SUS levels, probability route, lane groups (CTA family)
    kNumVariants
};

// Check-node route a variant computes (the item's DecodeArgs::method).
int variant_method(int v) {
    if (v >= kLevel16X && v <= kLevel256X) return kTensor;
    if ((v >= kGroup32T && v <= kGroup256T) || (v >= kLevel32T && v <= kLevel256T)) return kTransform;
    return kDirect;
}

int tensor_variant(int q) {
    switch (q) {
    case 16: return kLevel16X;
    case 32: return kLevel32X;
    case 64: return kLevel64X;
    case 128: return kLevel128X;
    case 256: return kLevel256X;
    }
    return -1;
}

__host__ __device__ constexpr bool cta_variant(int v) { return v >= kLevel2D; }

// CTA-family variants that work with a lane group per pair (q >= 32 and the
// tensor-core route): their CTAs take 256 threads.
__host__ __device__ constexpr bool lane_group_variant(int v) { return cta_variant(v) && !(v >= kLevel2D && v <= kLevel16D); }

// SUS CTA family: one frame per CTA, 256 threads when a transform-route item
// (a lane group per pair) is in the launch, else 128 (a thread per pair).

// Shared scratch per warp (floats) for the SUS variants.
constexpr int kWarpScratch = 3 * 256 + 4;  // the largest: group q=256 transform route, one group per warp

// Out-of-line variant bodies: each keeps its own register allocation instead
// of the union of all variants inlined into one kernel.
template <int Q>
__device__ __noinline__ void sus_team_call(const DecodeArgs& A, int f, const uint8_t* mul, const uint8_t* div,
                                           float* sa) {
    sus_team_frame<Q, 6>(A, f, mul, div, sa);
}

template <int Q, int METHOD>
__device__ __noinline__ void sus_group_call(const DecodeArgs& A, int f, const uint8_t* ex, const uint8_t* lg,
                                            float* sc) {
    sus_group_frame<Q, 6, 3, METHOD>(A, f, ex, lg, sc);
}

template <int Q, int METHOD>
__device__ __noinline__ void pus_call(const DecodeArgs& A, int f, const uint8_t* ex, const uint8_t* lg, float* sc) {
    pus_frame<Q, 6, 3, METHOD>(A, f, ex, lg, sc);
}

template <int Q, int T>
__device__ __noinline__ void sus_level_call(const DecodeArgs& A, int f, const uint8_t* mul, const uint8_t* div,
                                            float* dyn) {
    // batch items fold per visit (their options are the defaults, and the
    // running partials' scratch is not allocated for them)
    sus_level_frame<Q, 8, T, false>(A, f, mul, div, dyn, dyn + kLevelPiece * level_rs<Q>());
}

template <int Q, int T, int METHOD>
__device__ __noinline__ void sus_level_tr_call(const DecodeArgs& A, int f, const uint8_t* ex, const uint8_t* lg,
                                               float* dyn) {
    constexpr int G = Lay<Q>::G;
    float* sc = dyn + (size_t)level_tr_sub<Q>() * Q + (size_t)(threadIdx.x / G) * (Q + 4);
    sus_level_tr_frame<Q, T, METHOD>(A, f, ex, lg, dyn, sc);
}

template <int Q, int T>
__device__ __noinline__ void sus_level_tc_call(const DecodeArgs& A, int f, const uint8_t* ex, const uint8_t* lg,
                                               float* dyn) {
    sus_level_tc_frame<Q, T>(A, f, ex, lg, reinterpret_cast<uint8_t*>(dyn));
}

// Dynamic shared memory of a CTA-family variant with T threads.
template <int Q, int T>
constexpr size_t level_mixed_bytes() {
    return sizeof(float) * (Q <= 16 ? (size_t)(kLevelPiece + T) * level_rs<Q>()
                                    : (size_t)level_tr_sub<Q>() * Q + (size_t)(T / Lay<Q>::G) * (Q + 4));
}
constexpr size_t max2(size_t a, size_t b) { return a > b ? a : b; }

template <int T>
size_t cta_variant_smem(int v) {
    switch (v) {
    case kLevel2D: return level_mixed_bytes<2, T>();
    case kLevel4D: return level_mixed_bytes<4, T>();
    case kLevel8D: return level_mixed_bytes<8, T>();
    case kLevel16D: return level_mixed_bytes<16, T>();
    case kLevel32T: return level_mixed_bytes<32, T>();
    case kLevel64T: return level_mixed_bytes<64, T>();
    case kLevel128T: return level_mixed_bytes<128, T>();
    case kLevel256T: return level_mixed_bytes<256, T>();
    case kLevel32D: return level_mixed_bytes<32, T>();
    case kLevel64D: return level_mixed_bytes<64, T>();
    case kLevel128D: return level_mixed_bytes<128, T>();
    case kLevel256D: return level_mixed_bytes<256, T>();
    case kLevel16X: return TcLay<16, T>::total;
    case kLevel32X: return TcLay<32, T>::total;
    case kLevel64X: return TcLay<64, T>::total;
    case kLevel128X: return TcLay<128, T>::total;
    case kLevel256X: return TcLay<256, T>::total;
    }
    return 0;
}

template <int T>
constexpr size_t cta_smem_max() {
    return max2(max2(max2(TcLay<64, T>::total, TcLay<256, T>::total), max2(TcLay<128, T>::total, TcLay<32, T>::total)),
                max2(max2(level_mixed_bytes<256, T>(), level_mixed_bytes<64, T>()),
                     max2(level_mixed_bytes<16, T>(), TcLay<16, T>::total)));
}

// Index of the item holding global frame g (prefix sums, binary search).
__device__ __forceinline__ int find_item(const int* __restrict__ prefix, int n_items, int g) {
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Field tables for every q = 2^p the items use (items of equal q share the
// field polynomial): exp/log, and h a / h^-1 b for q <= 16.
struct FieldTables {
    uint8_t ex[8][512];
    uint8_t lg[8][256];
    uint8_t mul[4][256];   // q = 2, 4, 8, 16
    uint8_t div[4][256];
};

__device__ void load_fields(FieldTables& T, const DecodeArgs* items, const int* field_item, int tid, int nt) {
    for (int p = 0; p < 8; p++) {
        const int i = field_item[p];
        if (i < 0) continue;
        for (int x = tid; x < 512; x += nt) T.ex[p][x] = items[i].c.gexp[x];
        for (int x = tid; x < 256; x += nt) T.lg[p][x] = items[i].c.glog[x];
    }
    __syncthreads();
    if (field_item[0] >= 0) team_tables<2>(T.ex[0], T.lg[0], T.mul[0], T.div[0], tid, nt);
    if (field_item[1] >= 0) team_tables<4>(T.ex[1], T.lg[1], T.mul[1], T.div[1], tid, nt);
    if (field_item[2] >= 0) team_tables<8>(T.ex[2], T.lg[2], T.mul[2], T.div[2], tid, nt);
    if (field_item[3] >= 0) team_tables<16>(T.ex[3], T.lg[3], T.mul[3], T.div[3], tid, nt);
    __syncthreads();
}

__global__ void __launch_bounds__(kMixedThreads) k_sus_mixed(const DecodeArgs* __restrict__ items,
                                                             const int* __restrict__ prefix,
                                                             const int* __restrict__ variant, int n_items,
                                                             int total, int* counter, const int* field_item) {
    __shared__ __align__(16) FieldTables T;
    __shared__ __align__(16) float s_scr[(kMixedThreads / 32) * kWarpScratch];
    const int tid = threadIdx.x;
    load_fields(T, items, field_item, tid, blockDim.x);
    const int lane = tid & 31;
    float* wscr = s_scr + (tid / 32) * kWarpScratch;
    for (;;) {
        int gidx = 0;
        if (lane == 0) gidx = atomicAdd(counter, 1);
        gidx = __shfl_sync(0xffffffffu, gidx, 0);
        if (gidx >= total) break;
        const int it = find_item(prefix, n_items, gidx);
        const int f = gidx - __ldg(prefix + it);
        const DecodeArgs& A = items[it];
        const int pf = A.c.p - 1;
        const uint8_t* ex = T.ex[pf];
        const uint8_t* lg = T.lg[pf];
        const uint8_t* s_mul_it = T.mul[pf <= 3 ? pf : 0];
        const uint8_t* s_div_it = T.div[pf <= 3 ? pf : 0];
        const int var = __ldg(variant + it);
        if (cta_variant(var)) continue;   // decoded by the CTA-family kernel
        switch (var) {
        case kTeam4:
            if (lane < TeamLay<4>::TEAM)
                sus_team_call<4>(A, f, s_mul_it, s_div_it, wscr + (lane / TeamLay<4>::GS) * (2 * 4 + 4));
            break;
        case kTeam8:
            sus_team_call<8>(A, f, s_mul_it, s_div_it, wscr + (lane / TeamLay<8>::GS) * (2 * 8 + 4));
            break;
        case kTeam16:
            sus_team_call<16>(A, f, s_mul_it, s_div_it, wscr + (lane / TeamLay<16>::GS) * (2 * 16 + 4));
            break;
        case kGroup2D:
            if (lane < Lay<2>::G) sus_group_call<2, kDirect>(A, f, ex, lg, wscr);
            break;
        case kGroup4D:
            if (lane < Lay<4>::G) sus_group_call<4, kDirect>(A, f, ex, lg, wscr);
            break;
        case kGroup8D:
            if (lane < Lay<8>::G) sus_group_call<8, kDirect>(A, f, ex, lg, wscr);
            break;
        case kGroup16D:
            if (lane < Lay<16>::G) sus_group_call<16, kDirect>(A, f, ex, lg, wscr);
            break;
        case kGroup32T:
            if (lane < Lay<32>::G) sus_group_call<32, kTransform>(A, f, ex, lg, wscr);
            break;
        case kGroup64T:
            if (lane < Lay<64>::G) sus_group_call<64, kTransform>(A, f, ex, lg, wscr);
            break;
        case kGroup128T:
            if (lane < Lay<128>::G) sus_group_call<128, kTransform>(A, f, ex, lg, wscr);
            break;
        default:
            if (lane < Lay<256>::G) sus_group_call<256, kTransform>(A, f, ex, lg, wscr);
            break;
        }
        __syncwarp();
    }
}

// SUS, CTA family: one frame per CTA (level schedules).  With 256 threads
// (a lane-group variant present) three CTAs per SM, as the transform- and
// probability-route level kernels of q >= 32 reach on their own (80
// registers): those items hold most of a mixed batch's work, and two CTAs per
// SM (128 registers) left a third of their slots empty.
// With 512 threads (`MixedLaunch::wide`) one CTA per SM: twice the lane groups
// for each of fewer frames at once, for frames whose levels hold hundreds of
// pairs.
template <int NTH>
__global__ void __launch_bounds__(NTH, NTH == 512 ? 1 : (NTH == 256 ? 3 : 4)) k_sus_mixed_cta(const DecodeArgs* __restrict__ items,
                                                                    const int* __restrict__ prefix,
                                                                    const int* __restrict__ variant, int n_items,
                                                                    int total, int* counter, const int* field_item) {
    __shared__ __align__(16) FieldTables T;
    __shared__ int s_frame;
    extern __shared__ __align__(16) float s_dyn[];
    const int tid = threadIdx.x;
    load_fields(T, items, field_item, tid, blockDim.x);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_frame = atomicAdd(counter, 1);
        __syncthreads();
        const int gidx = s_frame;
        if (gidx >= total) break;
        const int it = find_item(prefix, n_items, gidx);
        const int var = __ldg(variant + it);
        if (!cta_variant(var)) continue;   // decoded by the warp-family kernel
        const int f = gidx - __ldg(prefix + it);
        const DecodeArgs& A = items[it];
        const int pf = A.c.p - 1;
        const uint8_t* ex = T.ex[pf];
        const uint8_t* lg = T.lg[pf];
        const uint8_t* mul = T.mul[pf <= 3 ? pf : 0];
        const uint8_t* div = T.div[pf <= 3 ? pf : 0];
        if constexpr (NTH == 512) {   // the wide form runs the FP32 lane-group variants only
            switch (var) {
            case kLevel32T: sus_level_tr_call<32, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
            case kLevel64T: sus_level_tr_call<64, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
            case kLevel128T: sus_level_tr_call<128, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
            case kLevel256T: sus_level_tr_call<256, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
            case kLevel32D: sus_level_tr_call<32, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
            case kLevel64D: sus_level_tr_call<64, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
            case kLevel128D: sus_level_tr_call<128, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
            case kLevel256D: sus_level_tr_call<256, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
            default: break;
            }
            continue;
        }
        switch (var) {
        case kLevel2D: sus_level_call<2, NTH>(A, f, mul, div, s_dyn); break;
        case kLevel4D: sus_level_call<4, NTH>(A, f, mul, div, s_dyn); break;
        case kLevel8D: sus_level_call<8, NTH>(A, f, mul, div, s_dyn); break;
        case kLevel16D: sus_level_call<16, NTH>(A, f, mul, div, s_dyn); break;
        case kLevel32T: sus_level_tr_call<32, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
        case kLevel64T: sus_level_tr_call<64, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
        case kLevel128T: sus_level_tr_call<128, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
        case kLevel256T: sus_level_tr_call<256, NTH, kTransform>(A, f, ex, lg, s_dyn); break;
        case kLevel32D: sus_level_tr_call<32, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
        case kLevel64D: sus_level_tr_call<64, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
        case kLevel128D: sus_level_tr_call<128, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
        case kLevel256D: sus_level_tr_call<256, NTH, kDirect>(A, f, ex, lg, s_dyn); break;
        case kLevel16X: sus_level_tc_call<16, NTH>(A, f, ex, lg, s_dyn); break;
        case kLevel32X: sus_level_tc_call<32, NTH>(A, f, ex, lg, s_dyn); break;
        case kLevel64X: sus_level_tc_call<64, NTH>(A, f, ex, lg, s_dyn); break;
        case kLevel128X: sus_level_tc_call<128, NTH>(A, f, ex, lg, s_dyn); break;
        case kLevel256X: sus_level_tc_call<256, NTH>(A, f, ex, lg, s_dyn); break;
        default: break;
        }
    }
}

// PUS: one CTA per frame, the item's q and check-node route pick the routine.
template <int Q>
constexpr int pus_mixed_scratch() { return (kPusThreads / Lay<Q>::G) * pus_group_scratch<Q, 6, kDirect>(); }
constexpr int imax(int a, int b) { return a > b ? a : b; }
// the largest over the variants (the probability route needs the most)
constexpr int kMixedPusScratch =
    imax(imax(imax(pus_mixed_scratch<2>(), pus_mixed_scratch<4>()), imax(pus_mixed_scratch<8>(), pus_mixed_scratch<16>())),
         imax(imax(pus_mixed_scratch<32>(), pus_mixed_scratch<64>()),
              imax(pus_mixed_scratch<128>(), pus_mixed_scratch<256>())));

__global__ void __launch_bounds__(kPusThreads) k_pus_mixed(const DecodeArgs* __restrict__ items,
                                                           const int* __restrict__ prefix, int n_items, int total,
                                                           int* counter, const int* field_item) {
    __shared__ __align__(16) FieldTables T;
    __shared__ int s_frame;
    extern __shared__ __align__(16) float s_scr[];
    const int tid = threadIdx.x;
    load_fields(T, items, field_item, tid, blockDim.x);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_frame = atomicAdd(counter, 1);
        __syncthreads();
        const int gidx = s_frame;
        if (gidx >= total) break;
        const int it = find_item(prefix, n_items, gidx);
        const int f = gidx - __ldg(prefix + it);
        const DecodeArgs& A = items[it];
        const uint8_t* ex = T.ex[A.c.p - 1];
        const uint8_t* lg = T.lg[A.c.p - 1];
        switch (A.c.q) {
        case 2: pus_call<2, kDirect>(A, f, ex, lg, s_scr); break;
        case 4: pus_call<4, kDirect>(A, f, ex, lg, s_scr); break;
        case 8: pus_call<8, kDirect>(A, f, ex, lg, s_scr); break;
        case 16: pus_call<16, kDirect>(A, f, ex, lg, s_scr); break;
        case 32:
            if (A.method == kDirect) pus_call<32, kDirect>(A, f, ex, lg, s_scr);
            else pus_call<32, kTransform>(A, f, ex, lg, s_scr);
            break;
        case 64:
            if (A.method == kDirect) pus_call<64, kDirect>(A, f, ex, lg, s_scr);
            else pus_call<64, kTransform>(A, f, ex, lg, s_scr);
            break;
        case 128:
            if (A.method == kDirect) pus_call<128, kDirect>(A, f, ex, lg, s_scr);
            else pus_call<128, kTransform>(A, f, ex, lg, s_scr);
            break;
        default:
            if (A.method == kDirect) pus_call<256, kDirect>(A, f, ex, lg, s_scr);
            else pus_call<256, kTransform>(A, f, ex, lg, s_scr);
            break;
        }
    }
}

int default_variant(int q) {
    switch (q) {
    case 2: return kLevel2D;
    case 4: return kLevel4D;
    case 8: return kLevel8D;
    case 16: return kLevel16D;
    case 32: return kLevel32D;
    case 64: return kLevel64D;
    case 128: return kLevel128T;
    default: return kLevel256T;
    }
}

// The variants of the route AUTO does not take for q >= 32: the transform
// route for q = 32, 64 (trading the probability route's relative precision
// for speed), the probability route for q = 128, 256 (exact, at q^2 FMAs per
// convolution).
std::vector<int> other_route_variants(int q) {
    switch (q) {
    case 32: return {kLevel32T, kGroup32T};
    case 64: return {kLevel64T, kGroup64T};
    case 128: return {kLevel128D};
    case 256: return {kLevel256D};
    }
    return {};
}

// SUS variants the autotuner may pick from (same check-node route, so the
// same results up to the order of rounding; level and team kernels of one q
// give the same bits).
std::vector<int> sus_candidates(int q) {
    switch (q) {
    case 2: return {kLevel2D, kGroup2D};
    case 4: return {kLevel4D, kTeam4, kGroup4D};
    case 8: return {kLevel8D, kTeam8, kGroup8D};
    case 16: return {kLevel16D, kTeam16, kGroup16D};
    case 32: return {kLevel32D};
    case 64: return {kLevel64D};
    case 128: return {kLevel128T, kGroup128T};
    default: return {kLevel256T, kGroup256T};
    }
}

int num_sms() { return device_sms(); }

// autotuner cache: (device, q, N, M, E, schedule) -> variant
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, long long, int>, int> g_tune;

std::tuple<int, int, int, int, long long, int> tune_key(const gfbp_code* c, int schedule) {
    int dev = 0;
    cudaGetDevice(&dev);
    return {dev, c->dev.q, c->dev.N, c->dev.M, c->dev.E, schedule};
}

}  // namespace
}  // namespace gfbp

namespace gfbp {

// Field-table owner per p (item index of the first item with q = 2^p), or an
// error when two codes of one q use different polynomials.
bool field_owners(const std::vector<const gfbp_code*>& codes, int* owner, std::string* why) {
    uint32_t poly[8] = {0};
    for (int p = 0; p < 8; p++) owner[p] = -1;
    for (size_t i = 0; i < codes.size(); i++) {
        const int pf = codes[i]->dev.p - 1;
        if (owner[pf] < 0) {
            owner[pf] = (int)i;
            poly[pf] = codes[i]->poly;
        } else if (poly[pf] != codes[i]->poly) {
            *why = "codes of the same field size must use the same field polynomial";
            return false;
        }
    }
    return true;
}

// Order of a launch's frame table: items with the costliest frames first (the
// frames are handed out in table order, so the longest decodes start first
// instead of setting the tail).  Cost of a frame ~ N q (work per sweep up to a
// log factor); ties keep the given order.
std::vector<int> heavy_first(const std::vector<const CodeDev*>& codes) {
    std::vector<int> order(codes.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)codes[a]->N * codes[a]->q > (long long)codes[b]->N * codes[b]->q;
    });
    return order;
}

void mixed_shape(MixedLaunch& m, const int* variants) {
    int occ = 1;
    if (m.schedule == GFBP_SUS) {
        m.has_cta = m.has_warp = false;
        m.cta_threads = 128;
        for (int i = 0; i < m.n_items; i++) {
            (cta_variant(variants[i]) ? m.has_cta : m.has_warp) = true;
            if (lane_group_variant(variants[i])) m.cta_threads = 256;
        }
        // the wide form when every CTA-family item is an FP32 lane-group variant
        bool wide = m.wide && m.cta_threads == 256;
        for (int i = 0; i < m.n_items && wide; i++)
            if (cta_variant(variants[i])) wide = lane_group_variant(variants[i]) && variant_method(variants[i]) != kTensor;
        if (wide) m.cta_threads = 512;
        m.cta_smem = 0;
        for (int i = 0; i < m.n_items; i++)
            m.cta_smem = max2(m.cta_smem, m.cta_threads == 512   ? cta_variant_smem<512>(variants[i])
                                          : m.cta_threads == 256 ? cta_variant_smem<256>(variants[i])
                                                                 : cta_variant_smem<128>(variants[i]));
        kernel_prepare((const void*)k_sus_mixed, kMixedThreads, 0, &occ);
        const long long want = ((long long)m.total + 3) / 4;
        const long long cap = (long long)num_sms() * (occ > 0 ? occ : 1);
        m.grid = (int)(want < cap ? want : cap);
        int occ2 = 1;
        if (m.cta_threads == 512)
            kernel_prepare((const void*)k_sus_mixed_cta<512>, 512, m.cta_smem, &occ2);
        else if (m.cta_threads == 256)
            kernel_prepare((const void*)k_sus_mixed_cta<256>, 256, m.cta_smem, &occ2);
        else
            kernel_prepare((const void*)k_sus_mixed_cta<128>, 128, m.cta_smem, &occ2);
        const long long cap2 = (long long)num_sms() * (occ2 > 0 ? occ2 : 1);
        m.grid_cta = (int)(m.total < cap2 ? m.total : cap2);
    } else {
        m.pus_smem = sizeof(float) * (size_t)kMixedPusScratch;
        kernel_prepare((const void*)k_pus_mixed, kPusThreads, m.pus_smem, &occ);
        const long long cap = (long long)num_sms() * (occ > 0 ? occ : 1);
        m.grid = (int)(m.total < cap ? m.total : cap);
    }
}

cudaError_t mixed_launch(const MixedLaunch& m, cudaStream_t s) {
    if (m.total == 0 || m.grid == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(m.d_counter, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (m.schedule == GFBP_SUS) {
        if (m.has_cta)
        {
            if (m.cta_threads == 512)
                k_sus_mixed_cta<512><<<m.grid_cta, 512, m.cta_smem, s>>>(m.d_args, m.d_prefix, m.d_variant, m.n_items,
                                                                        m.total, m.d_counter + 1, m.d_field);
            else if (m.cta_threads == 256)
                k_sus_mixed_cta<256><<<m.grid_cta, 256, m.cta_smem, s>>>(m.d_args, m.d_prefix, m.d_variant, m.n_items,
                                                                        m.total, m.d_counter + 1, m.d_field);
            else
                k_sus_mixed_cta<128><<<m.grid_cta, 128, m.cta_smem, s>>>(m.d_args, m.d_prefix, m.d_variant, m.n_items,
                                                                        m.total, m.d_counter + 1, m.d_field);
        }
        if (m.has_warp)
            k_sus_mixed<<<m.grid, kMixedThreads, 0, s>>>(m.d_args, m.d_prefix, m.d_variant, m.n_items, m.total,
                                                         m.d_counter, m.d_field);
    } else
        k_pus_mixed<<<m.grid, kPusThreads, m.pus_smem, s>>>(m.d_args, m.d_prefix, m.n_items, m.total, m.d_counter,
                                                            m.d_field);
    return cudaGetLastError();
}

int tuned_variant(const gfbp_code* code, int schedule) {
    int v = default_variant(code->dev.q);
    if (schedule == GFBP_SUS) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto f = g_tune.find(tune_key(code, schedule));
        if (f != g_tune.end()) v = f->second;
    }
    return v;
}

}  // namespace gfbp

struct gfbp_batch {
    std::vector<gfbp::DecodeArgs> args;   // caller's item order
    std::vector<int> variant;             // caller's item order
    std::vector<int> order;               // frame-table position -> caller's item
    void* dmem = nullptr;  // items | prefix | variants | counter | field owners | per-item workspaces
    gfbp::MixedLaunch m;
};

using namespace gfbp;

namespace {

// The device frame table in b->order: items, frame prefix, variants, field
// owners (synchronous).
cudaError_t upload_tables(gfbp_batch* b) {
    const int n = (int)b->args.size();
    std::vector<DecodeArgs> a(n);
    std::vector<int> prefix(n + 1, 0), v(n);
    int owner[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    for (int k = 0; k < n; k++) {
        const int i = b->order[k];
        a[k] = b->args[i];
        v[k] = b->variant[i];
        prefix[k + 1] = prefix[k] + a[k].F;
        const int pf = a[k].c.p - 1;
        if (owner[pf] < 0) owner[pf] = k;
    }
    cudaError_t e = cudaMemcpy(b->m.d_args, a.data(), sizeof(DecodeArgs) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->m.d_prefix, prefix.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->m.d_variant, v.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->m.d_field, owner, sizeof(owner), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

extern "C" gfbp_status gfbp_batch_create(const gfbp_batch_item* items, int32_t n_items, gfbp_schedule schedule,
                                         int32_t max_iter, const gfbp_options* options, gfbp_batch** out) {
    if (!out || !items || n_items < 1 || n_items > kMaxItems) {
        set_error("gfbp_batch_create: need 1 <= n_items <= 65536 items and an output handle");
        return GFBP_EINVAL;
    }
    *out = nullptr;
    if (schedule != GFBP_PUS && schedule != GFBP_SUS) { set_error("gfbp_batch_create: unknown schedule"); return GFBP_EINVAL; }
    if (max_iter < 1) { set_error("gfbp_batch_create: max_iter must be >= 1"); return GFBP_EINVAL; }
    if (options && (options->syndrome || options->punct || options->xhat_trace || options->post)) {
        set_error("gfbp_batch_create: per-call options (syndrome, punct, trace, post) are not taken by batches");
        return GFBP_EUNSUPPORTED;
    }
    std::vector<size_t> ws(n_items);
    std::vector<int> prefix(n_items + 1, 0);
    std::vector<const gfbp_code*> codes(n_items);
    for (int i = 0; i < n_items; i++) {
        const gfbp_batch_item& it = items[i];
        if (!it.code || it.n_frames < 0 || (it.n_frames > 0 && (!it.obs || !it.x_hat || !it.iters || !it.converged))) {
            set_error("gfbp_batch_create: item " + std::to_string(i) + " has a NULL code, input or output");
            return GFBP_EINVAL;
        }
        if (it.code->dev.dcmax > 6 || it.code->dev.dvmax > 3) {
            set_error("gfbp_batch_create: item " + std::to_string(i) +
                      ": batched kernels take row degree <= 6 and column degree <= 3");
            return GFBP_EUNSUPPORTED;
        }
        gfbp_status st = gfbp_workspace_size(it.code, it.n_frames, schedule, it.prior, 0, &ws[i]);
        if (st != GFBP_OK) return st;
        prefix[i + 1] = prefix[i] + it.n_frames;
        codes[i] = it.code;
    }
    int owner[8];
    std::string why;
    if (!field_owners(codes, owner, &why)) {
        set_error("gfbp_batch_create: " + why);
        return GFBP_EUNSUPPORTED;
    }
    gfbp_batch* b = new (std::nothrow) gfbp_batch();
    if (!b) { set_error("gfbp_batch_create: out of host memory"); return GFBP_ENOMEM; }
    const size_t a_args = (sizeof(DecodeArgs) * n_items + 255) & ~(size_t)255;
    const size_t a_int = (sizeof(int) * (n_items + 1) + 255) & ~(size_t)255;
    size_t total = a_args + 2 * a_int + 512;
    std::vector<size_t> ws_off(n_items);
    for (int i = 0; i < n_items; i++) { ws_off[i] = total; total += (ws[i] + 255) & ~(size_t)255; }
    cudaError_t e = cudaMalloc(&b->dmem, total);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_batch_create: ") + cudaGetErrorString(e));
        delete b;
        return e == cudaErrorMemoryAllocation ? GFBP_ENOMEM : GFBP_ECUDA;
    }
    uint8_t* base = static_cast<uint8_t*>(b->dmem);
    MixedLaunch& m = b->m;
    m.d_args = reinterpret_cast<DecodeArgs*>(base);
    m.d_prefix = reinterpret_cast<int*>(base + a_args);
    m.d_variant = reinterpret_cast<int*>(base + a_args + a_int);
    m.d_counter = reinterpret_cast<int*>(base + a_args + 2 * a_int);
    m.d_field = reinterpret_cast<int*>(base + a_args + 2 * a_int + 256);
    m.n_items = n_items;
    m.total = prefix[n_items];
    m.schedule = schedule;
    b->args.resize(n_items);
    b->variant.resize(n_items);
    for (int i = 0; i < n_items; i++) {
        const gfbp_batch_item& it = items[i];
        const int q = it.code->dev.q;
        const int method = q <= kAutoDirectMaxQ ? kDirect : kTransform;
        e = batch_prepare_item(b->args[i], base + ws_off[i], it.code, it.n_frames, it.obs, it.channel, schedule,
                               it.prior, max_iter, it.x_hat, it.iters, it.converged, nullptr, method, nullptr, 0);
        if (e != cudaSuccess) {
            cudaFree(b->dmem);
            delete b;
            return GFBP_EINVAL;
        }
        b->variant[i] = tuned_variant(it.code, schedule);
    }
    {
        std::vector<const CodeDev*> cd(n_items);
        for (int i = 0; i < n_items; i++) cd[i] = &items[i].code->dev;
        b->order = heavy_first(cd);
    }
    e = upload_tables(b);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_batch_create: ") + cudaGetErrorString(e));
        cudaFree(b->dmem);
        delete b;
        return GFBP_ECUDA;
    }
    mixed_shape(m, b->variant.data());
    *out = b;
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_batch_run(gfbp_batch* b, void* stream_v) {
    if (!b) { set_error("gfbp_batch_run: NULL batch"); return GFBP_EINVAL; }
    cudaStream_t s = static_cast<cudaStream_t>(stream_v);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < b->args.size() && e == cudaSuccess; i++) {
        const DecodeArgs& A = b->args[i];
        if (A.F == 0) continue;
        e = launch_channel(A, s);
        if (e == cudaSuccess && A.markov) e = launch_fill_prior(A, s);
        if (e == cudaSuccess && b->m.schedule == GFBP_SUS) e = launch_init_dev(A, s);
    }
    if (e == cudaSuccess) e = mixed_launch(b->m, s);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_batch_run: ") + cudaGetErrorString(e));
        return GFBP_ECUDA;
    }
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_batch_variants(const gfbp_batch* b, int32_t* variants) {
    if (!b || !variants) { set_error("gfbp_batch_variants: NULL argument"); return GFBP_EINVAL; }
    for (size_t i = 0; i < b->variant.size(); i++) variants[i] = b->variant[i];
    return GFBP_OK;
}

extern "C" gfbp_status gfbp_batch_set_variants(gfbp_batch* b, const int32_t* variants) {
    if (!b || !variants) { set_error("gfbp_batch_set_variants: NULL argument"); return GFBP_EINVAL; }
    const int n = (int)b->variant.size();
    std::vector<int> v(n);
    for (int i = 0; i < n; i++) {
        const int q = b->args[i].c.q;
        std::vector<int> ok = b->m.schedule == GFBP_SUS ? sus_candidates(q) : std::vector<int>{default_variant(q)};
        if (b->m.schedule == GFBP_SUS && tensor_variant(q) >= 0) ok.push_back(tensor_variant(q));
        if (b->m.schedule == GFBP_SUS)
            for (int t : other_route_variants(q)) ok.push_back(t);
        bool found = false;
        for (int c : ok) found |= (c == variants[i]);
        if (!found) {
            set_error("gfbp_batch_set_variants: variant " + std::to_string(variants[i]) + " cannot decode item " +
                      std::to_string(i) + " (q = " + std::to_string(q) + ")");
            return GFBP_EINVAL;
        }
        v[i] = variants[i];
    }
    // a variant of another check-node route changes the stored message form
    // (and the initialisation kernel of gfbp_batch_run)
    for (int i = 0; i < n; i++) b->args[i].method = variant_method(v[i]);
    b->variant = v;
    cudaError_t e = upload_tables(b);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_batch_set_variants: ") + cudaGetErrorString(e));
        return GFBP_ECUDA;
    }
    mixed_shape(b->m, b->variant.data());
    return GFBP_OK;
}

extern "C" void gfbp_batch_destroy(gfbp_batch* b) {
    if (!b) return;
    cudaFree(b->dmem);
    delete b;
}

extern "C" gfbp_status gfbp_autotune(const gfbp_code* code, int32_t n_frames, const float* obs, gfbp_channel channel,
                                     gfbp_schedule schedule, const gfbp_prior* prior, int32_t max_iter, void* stream_v,
                                     int32_t* chosen) {
    if (!code || !obs || n_frames < 1 || !chosen) {
        set_error("gfbp_autotune: need a code, n_frames >= 1 frames of obs and an output");
        return GFBP_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_v);
    const std::vector<int> cand = schedule == GFBP_SUS ? sus_candidates(code->dev.q)
                                                       : std::vector<int>{default_variant(code->dev.q)};
    void* out = nullptr;
    const size_t N = (size_t)code->dev.N;
    cudaError_t e = cudaMalloc(&out, (size_t)n_frames * (N + 2 * sizeof(int)) + 256);
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_autotune: ") + cudaGetErrorString(e));
        return GFBP_ENOMEM;
    }
    uint8_t* x_hat = static_cast<uint8_t*>(out);
    int32_t* iters = reinterpret_cast<int32_t*>(x_hat + (((size_t)n_frames * N + 15) & ~(size_t)15));
    uint8_t* conv = reinterpret_cast<uint8_t*>(iters + n_frames);
    gfbp_batch_item item{code, n_frames, obs, channel, prior, x_hat, iters, conv};
    gfbp_batch* b = nullptr;
    gfbp_status st = gfbp_batch_create(&item, 1, schedule, max_iter, nullptr, &b);
    if (st != GFBP_OK) { cudaFree(out); return st; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best = cand[0];
    for (int v : cand) {
        b->variant[0] = v;
        e = cudaMemcpy(b->m.d_variant, &v, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        mixed_shape(b->m, b->variant.data());
        float ms = 0.f;
        for (int rep = 0; rep < 3 && st == GFBP_OK; rep++) {   // first run warms up
            cudaEventRecord(e0, s);
            st = gfbp_batch_run(b, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;
        }
        if (st != GFBP_OK) break;
        if (ms < best_ms) { best_ms = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gfbp_batch_destroy(b);
    cudaFree(out);
    if (st != GFBP_OK) return st;
    if (e != cudaSuccess) {
        set_error(std::string("gfbp_autotune: ") + cudaGetErrorString(e));
        return GFBP_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[tune_key(code, schedule)] = best;
    }
    *chosen = best;
    return GFBP_OK;
}
