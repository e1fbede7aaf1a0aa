// sai.cu -- construction of the sparse approximate inverse M ~ A~^{-1}
// (section 2 of the paper): n independent problems min ||A~ m_k - e_k||
// (eq. (subprob)) reduced to min ||A^_k m^_k - e^_k|| (eq. (lsprob)) and solved
// by Householder QR, one lane group per column.
//
// Per column k a group of G lanes (G = 8, 16 or 32: four, two or one column
// per warp) keeps, in a private workspace:
//   S      the pattern (insertion order), |S| <= SCAP
//   L      the rows of A~(:,S) plus k (row k always at local position 0),
//          with a hash row -> local position, |L| <= LCAP
//   Q      A^ = A~(L,S) factored in place: Householder vectors below and on
//          the diagonal, R above it (column-major, leading dimension LCAP),
//          rdiag = diag(R), beta = 2/(v^T v)
//   cv     Q^T e^,   m  the LS solution,   r  the residual A^ m - e^ on L
// When S grows, only the new columns are gathered: the old reflectors are
// applied to them and the trailing block is factored ("updating m^_k instead of
// resolving it", section 2.1). New rows are zero in the old columns because L
// already holds every nonzero row of A~(:,S_old).
//
// SPAI (section 2.1): candidates N \ S from the rows of L (CSR of A~),
// rho_j^2 = ||r||^2 - (r^T A~e_j)^2/||A~e_j||^2 (eq. (rhoj)), ranked by the key
// (floor(rho_j^2/||r||^2 * 2^key_bits) << 32 | j) and the mn smallest added;
// rho_j^2/||r||^2 is formed as 1 - (r^T A~e_j)^2 ||A~e_j||^-2 ||r||^-2 with the
// reciprocals taken once per column of A~ and once per loop.
// PSAI(tol) (section 2.2): drop |m_jk| <= tol_k (eq. (tolk)); grow
// S^(l+1) = P(|A~| a^(l)) u S_kept.
//
// Workspace tiers: the first runs in shared memory with a small workspace
// (|L| <= 32, |S| <= 8) and 8- or 16-lane groups, for the columns of stencil
// matrices whose patterns stay small; tier 0 in shared memory with one
// column per warp; a column that outgrows a tier is queued and restarted in
// the next: tier 0, then the global-memory tiers 1, 2 and 3 (tier 3 for
// columns whose rows reach more than 4096 candidate columns, as in
// heavy-tailed matrices). A restart reproduces the column's steps; the
// rounding of its sums depends on the group size, so a column's result
// depends on the tier that finishes it, which the column alone decides.
#include <float.h>

#include <mutex>

#include "internal.h"

namespace {

enum { ST_DONE = 0, ST_OVERFLOW = 1, ST_SINGULAR = 2 };

// Algorithmic bytes of the build (site PROF_SAI_BUILD), per finished column:
// the final pattern's columns read (12 B per stored entry), the row patterns
// of L read for candidates (4 B per entry) and the column written (12 B per entry).
// Flops: d_swork holds the FP64 ones, d_swork32 the FP32 ones (the QR of
// the refined form).
__device__ double d_swork[PROF_NSITES * 2];
__device__ double d_swork32;
constexpr int MNMAX = 8;

struct SaiMat {
    int32_t n;
    const int64_t* __restrict__ cp;  // CSC of A~
    const int32_t* __restrict__ ri;
    const double* __restrict__ cv;
    const int64_t* __restrict__ rp;  // CSR pattern of A~
    const int32_t* __restrict__ rc;
    const double* __restrict__ icn;  // 1/||A~e_j||^2 (0 for an empty column)
    double norm1;
};

struct SpaiArgs {
    double delta;
    double scale;  // 2^key_bits
    int mn, max_aug;
};

struct PsaiArgs {
    double delta, tol;
    int tol_mode, lmax;
    int lfill;   // tol_mode 2
    int growth;  // 0: reading (A); 1: reading (C), dropped positions stay dropped
};

struct Out {
    int32_t smax;      // output slots per column
    int32_t* cnt;      // [n]
    int32_t* rows;     // [n * smax]
    double* vals;      // [n * smax]
    int32_t* loops;    // [n]
    double* res;       // [n]
    double* res_post;  // [n] (PSAI)
    int32_t* tier;     // [n] tier that finished the column
    // the large-pattern tier writes its columns to slots of its own (the
    // column's index in that tier's work list): big_slot[k] >= 0 marks them
    int32_t big_smax;  // slots per large column (0: not the large tier)
    int32_t* big_slot; // [n], -1 for the other columns
    int32_t* big_rows; // [work list length * big_smax]
    double* big_vals;
};

constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

template <int LCAP_, int SCAP_, int HL_, int HC_, class TQ_ = double>
struct Tier {
    using TQ = TQ_;  // scalar of the QR factors (double, or float for the refined form)
    static constexpr int LCAP = LCAP_, SCAP = SCAP_, HL = HL_, HC = HC_;
    static constexpr size_t OFF_Q = 0;
    static constexpr size_t OFF_CV = OFF_Q + sizeof(TQ) * LCAP * SCAP;
    static constexpr size_t OFF_R = a16(OFF_CV + sizeof(TQ) * LCAP);
    static constexpr size_t OFF_M = OFF_R + 8ull * LCAP;
    static constexpr size_t OFF_G = OFF_M + 8ull * SCAP;
    static constexpr size_t OFF_BETA = OFF_G + 8ull * SCAP;
    static constexpr size_t OFF_RD = OFF_BETA + sizeof(TQ) * SCAP;
    static constexpr size_t OFF_LROW = a16(OFF_RD + sizeof(TQ) * SCAP);
    static constexpr size_t OFF_HK = OFF_LROW + 4ull * LCAP;
    static constexpr size_t OFF_HV = OFF_HK + 4ull * HL;
    static constexpr size_t OFF_S = OFF_HV + 4ull * HL;
    static constexpr size_t OFF_A0 = OFF_S + 4ull * SCAP;
    static constexpr size_t OFF_A1 = OFF_A0 + 4ull * SCAP;
    static constexpr size_t OFF_CK = OFF_A1 + 4ull * SCAP;
    static constexpr size_t OFF_CF = OFF_CK + 4ull * HC;
    static constexpr size_t OFF_KP = OFF_CF + (size_t)HC;
    static constexpr size_t BYTES = a16(OFF_KP + (size_t)SCAP);
    // distance between the workspaces of consecutive groups: a multiple of
    // 128 bytes plus 32, so that the 8-lane groups of one warp start in
    // different shared-memory banks
    static constexpr size_t STRIDE = ((BYTES + 127) & ~size_t(127)) + 32;
    static_assert(HL >= 2 * LCAP && (HL & (HL - 1)) == 0, "row hash");
    static_assert(HC >= 2 * SCAP && (HC & (HC - 1)) == 0, "candidate hash");
};

using TierS = Tier<32, 8, 64, 128>;         // shared memory, small patterns, ~4.1 KB per group
using Tier0 = Tier<64, 16, 128, 512>;      // shared memory, ~13.7 KB per warp
using Tier1 = Tier<256, 64, 512, 2048>;    // global memory, ~150 KB per warp
using Tier2 = Tier<1024, 128, 2048, 8192>; // global memory, ~1.1 MB per warp
using Tier3 = Tier<2048, 128, 4096, 65536>; // global memory, ~2.4 MB per warp (up to 32768 candidates)
using Tier4 = Tier<4096, 2048, 8192, 65536>; // global memory, ~68 MB per warp: the large-pattern tier
using TierSF = Tier<32, 8, 64, 128, float>;
using Tier0F = Tier<64, 16, 128, 512, float>;
using Tier1F = Tier<256, 64, 512, 2048, float>;
using Tier2F = Tier<1024, 128, 2048, 8192, float>;
using Tier3F = Tier<2048, 128, 4096, 65536, float>;
using Tier4F = Tier<4096, 2048, 8192, 65536, float>;

// Every loop of the device code below whose trip count is not a small
// constant is kept rolled (#pragma unroll 1): the build is bound by
// instruction fetch (its warps run different steps of different columns at
// once), and unrolled copies of the hash probes and of the per-column step
// loops at every inlined call site push its code out of the instruction
// cache (64^3 SPAI: 11.8 ms unrolled, 6.7 ms rolled).

// The lanes that work on one column: a group of G consecutive lanes of a
// warp (G = 32: the whole warp). Every reduction, vote and barrier below is
// over the group only, so the groups of a warp run independent columns.
template <int G>
struct Grp {
    static_assert(G == 8 || G == 16 || G == 32, "group size");
    unsigned mask;  // the group's lanes within the warp
    int base;       // first lane of the group
    int l;          // lane within the group
    __device__ __forceinline__ Grp()
    {
        const int lane = threadIdx.x & 31;
        l = lane & (G - 1);
        base = lane & ~(G - 1);
        mask = G == 32 ? 0xffffffffu : (((1u << (G & 31)) - 1u) << base);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    // the predicate's votes of the group, bit i = group lane i
    __device__ __forceinline__ unsigned ballot(bool p) const
    {
        const unsigned b = __ballot_sync(mask, p);
        return G == 32 ? b : (b >> base) & ((1u << (G & 31)) - 1u);
    }
    __device__ __forceinline__ bool any(bool p) const { return __any_sync(mask, p); }
    template <class V>
    __device__ __forceinline__ V bcast(V v, int src) const
    {
        return __shfl_sync(mask, v, base + src);
    }
    // butterfly sum over the group (for G = 32 the order of warp_sum)
    template <class V>
    __device__ __forceinline__ V sum(V v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
        return v;
    }
    __device__ __forceinline__ unsigned long long min_u64(unsigned long long v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(mask, v, o);
            v = w < v ? w : v;
        }
        return v;
    }
};

template <class TQ>
struct WsT {
    TQ *Q, *cv, *beta, *rd;  // QR factors, Q^T e^, 2/(v^T v), diag(R)
    double *r, *m, *g;       // FP64 residual, solution, refinement scratch
    int32_t *Lrow, *hk, *hv, *S, *a0, *a1, *ck;
    uint8_t *cf, *kp;
};

template <class T>
__device__ __forceinline__ WsT<typename T::TQ> bind_ws(char* b)
{
    using TQ = typename T::TQ;
    WsT<TQ> w;
    w.Q = (TQ*)(b + T::OFF_Q);
    w.cv = (TQ*)(b + T::OFF_CV);
    w.r = (double*)(b + T::OFF_R);
    w.m = (double*)(b + T::OFF_M);
    w.g = (double*)(b + T::OFF_G);
    w.beta = (TQ*)(b + T::OFF_BETA);
    w.rd = (TQ*)(b + T::OFF_RD);
    w.Lrow = (int32_t*)(b + T::OFF_LROW);
    w.hk = (int32_t*)(b + T::OFF_HK);
    w.hv = (int32_t*)(b + T::OFF_HV);
    w.S = (int32_t*)(b + T::OFF_S);
    w.a0 = (int32_t*)(b + T::OFF_A0);
    w.a1 = (int32_t*)(b + T::OFF_A1);
    w.ck = (int32_t*)(b + T::OFF_CK);
    w.cf = (uint8_t*)(b + T::OFF_CF);
    w.kp = (uint8_t*)(b + T::OFF_KP);
    return w;
}

__device__ __forceinline__ uint32_t hmix(int32_t key)
{
    uint32_t h = (uint32_t)key;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Lookup in an open-addressing table (keys -1 = empty). Returns the value or -1.
template <int H>
__device__ __forceinline__ int32_t hfind(const int32_t* hk, const int32_t* hv, int32_t key)
{
    uint32_t s = hmix(key) & (H - 1);
#pragma unroll 1
    for (int probe = 0; probe < H; ++probe) {
        int32_t k = hk[s];
        if (k == key) return hv[s];
        if (k == -1) return -1;
        s = (s + 1) & (H - 1);
    }
    return -1;
}

// Slot of key (inserting it if absent); -1 if the table is full.
template <int H>
__device__ __forceinline__ int hinsert(int32_t* hk, int32_t key, bool& inserted)
{
    uint32_t s = hmix(key) & (H - 1);
    inserted = false;
#pragma unroll 1
    for (int probe = 0; probe < H; ++probe) {
        int32_t k = *((volatile int32_t*)&hk[s]);
        if (k == key) return (int)s;
        if (k == -1) {
            int32_t old = atomicCAS(&hk[s], -1, key);
            if (old == -1) {
                inserted = true;
                return (int)s;
            }
            if (old == key) return (int)s;
        }
        s = (s + 1) & (H - 1);
    }
    return -1;
}

template <int H>
__device__ __forceinline__ int hslot(const int32_t* hk, int32_t key)
{
    uint32_t s = hmix(key) & (H - 1);
#pragma unroll 1
    for (int probe = 0; probe < H; ++probe) {
        int32_t k = hk[s];
        if (k == key) return (int)s;
        if (k == -1) return -1;
        s = (s + 1) & (H - 1);
    }
    return -1;
}

// Adds the rows of column j of A~ to L. New rows get consecutive positions in
// entry order, so L's order does not depend on scheduling. False on overflow.
template <class T, int G>
__device__ bool add_rows(const WsT<typename T::TQ>& w, const SaiMat& A, int32_t j, int& nL)
{
    const Grp<G> g;
    const int64_t b = A.cp[j], e = A.cp[j + 1];
#pragma unroll 1
    for (int64_t base = b; base < e; base += G) {
        const int64_t q = base + g.l;
        bool isnew = false;
        int slot = 0;
        int32_t i = -1;
        if (q < e) {
            i = A.ri[q];
            slot = hinsert<T::HL>(w.hk, i, isnew);
        }
        if (g.any(slot < 0)) return false;
        const unsigned mask = g.ballot(isnew);
        const int cnt = __popc(mask);
        if (nL + cnt > T::LCAP) return false;
        if (isnew) {
            const int pos = nL + __popc(mask & ((1u << g.l) - 1u));
            w.hv[slot] = pos;
            w.Lrow[pos] = i;
        }
        nL += cnt;
        g.sync();
    }
    return true;
}

// Resets the per-column state to S = {k}, L = {k}, cv = e^.
template <class T, int G>
__device__ void col_init(const WsT<typename T::TQ>& w, int32_t k, int& nL, int& nS, int& nfact)
{
    const Grp<G> g;
#pragma unroll 1
    for (int q = g.l; q < T::HL; q += G) w.hk[q] = -1;
    g.sync();
    if (g.l == 0) {
        bool ins;
        int sl = hinsert<T::HL>(w.hk, k, ins);
        w.hv[sl] = 0;
        w.Lrow[0] = k;
        w.cv[0] = 1;
    }
    g.sync();
    nL = 1;
    nS = 1;
    nfact = 0;
}

// Gathers the new columns S[nfact..nS), updates the QR factorisation and
// solves R m = (Q^T e^)(0:nS). Returns ST_DONE, ST_OVERFLOW or ST_SINGULAR.
template <class T, int G>
__device__ int ls_update(const WsT<typename T::TQ>& w, const SaiMat& A, int& nL, int nS, int& nfact)
{
    using TQ = typename T::TQ;
    const Grp<G> g;
    const int nL_old = nL;
#pragma unroll 1
    for (int t = nfact; t < nS; ++t)
        if (!add_rows<T, G>(w, A, w.S[t], nL)) return ST_OVERFLOW;
    // zero the new rows of the old columns and of cv, and the new columns
#pragma unroll 1
    for (int t = 0; t < nS; ++t) {
        TQ* col = w.Q + (size_t)t * T::LCAP;
#pragma unroll 1
        for (int i = (t < nfact ? nL_old : 0) + g.l; i < nL; i += G) col[i] = 0;
    }
#pragma unroll 1
    for (int i = nL_old + g.l; i < nL; i += G) w.cv[i] = 0;
    g.sync();
#pragma unroll 1
    for (int t = nfact; t < nS; ++t) {
        const int32_t j = w.S[t];
        TQ* col = w.Q + (size_t)t * T::LCAP;
#pragma unroll 1
        for (int64_t q = A.cp[j] + g.l; q < A.cp[j + 1]; q += G) {
            const int pos = hfind<T::HL>(w.hk, w.hv, A.ri[q]);
            if (pos >= 0) col[pos] = (TQ)A.cv[q];
        }
    }
    g.sync();
    // old reflectors on the new columns
#pragma unroll 1
    for (int jr = 0; jr < nfact; ++jr) {
        const TQ* v = w.Q + (size_t)jr * T::LCAP;
        const TQ bj = w.beta[jr];
#pragma unroll 1
        for (int t = nfact; t < nS; ++t) {
            TQ* col = w.Q + (size_t)t * T::LCAP;
            TQ d = 0;
#pragma unroll 1
            for (int i = jr + g.l; i < nL; i += G) d = fma(v[i], col[i], d);
            d = g.sum(d);
            const TQ f = bj * d;
#pragma unroll 1
            for (int i = jr + g.l; i < nL; i += G) col[i] = fma(-f, v[i], col[i]);
            g.sync();
        }
    }
    // factor the trailing block column by column
#pragma unroll 1
    for (int t = nfact; t < nS; ++t) {
        TQ* col = w.Q + (size_t)t * T::LCAP;
        TQ s2 = 0;
#pragma unroll 1
        for (int i = t + g.l; i < nL; i += G) s2 = fma(col[i], col[i], s2);
        s2 = g.sum(s2);
        if (!(s2 > (TQ)0)) return ST_SINGULAR;
        const TQ nrm = sqrt(s2);
        const TQ x0 = col[t];
        const TQ alpha = x0 >= (TQ)0 ? -nrm : nrm;
        const TQ bt = (TQ)1 / (nrm * (nrm + fabs(x0)));  // 2/(v^T v), v^T v = 2 nrm (nrm + |x0|)
        g.sync();
        if (g.l == 0) {
            col[t] = x0 - alpha;
            w.rd[t] = alpha;
            w.beta[t] = bt;
        }
        g.sync();
#pragma unroll 1
        for (int t2 = t + 1; t2 <= nS; ++t2) {
            TQ* c2 = t2 < nS ? w.Q + (size_t)t2 * T::LCAP : w.cv;
            TQ d = 0;
#pragma unroll 1
            for (int i = t + g.l; i < nL; i += G) d = fma(col[i], c2[i], d);
            d = g.sum(d);
            const TQ f = bt * d;
#pragma unroll 1
            for (int i = t + g.l; i < nL; i += G) c2[i] = fma(-f, col[i], c2[i]);
            g.sync();
        }
    }
    nfact = nS;
    // back substitution (FP64 arithmetic on the stored factors)
#pragma unroll 1
    for (int i = g.l; i < nS; i += G) w.m[i] = (double)w.cv[i];
    g.sync();
#pragma unroll 1
    for (int t = nS - 1; t >= 0; --t) {
        const double mt = w.m[t] / (double)w.rd[t];
        g.sync();
        if (g.l == 0) w.m[t] = mt;
        const TQ* col = w.Q + (size_t)t * T::LCAP;
#pragma unroll 1
        for (int i = g.l; i < t; i += G) w.m[i] = fma(-(double)col[i], mt, w.m[i]);
        g.sync();
    }
    return ST_DONE;
}

// r = A~(L,S) m - e^ on L (only the columns with use[t] != 0 when use given);
// returns ||r||^2.
template <class T, int G>
__device__ double residual(const WsT<typename T::TQ>& w, const SaiMat& A, int nL, int nS, const uint8_t* use)
{
    const Grp<G> g;
#pragma unroll 1
    for (int i = g.l; i < nL; i += G) w.r[i] = (i == 0) ? -1.0 : 0.0;
    g.sync();
#pragma unroll 1
    for (int t = 0; t < nS; ++t) {
        if (use && !use[t]) continue;
        const int32_t j = w.S[t];
        const double mt = w.m[t];
#pragma unroll 1
        for (int64_t q = A.cp[j] + g.l; q < A.cp[j + 1]; q += G) {
            const int pos = hfind<T::HL>(w.hk, w.hv, A.ri[q]);
            if (pos >= 0) w.r[pos] = fma(A.cv[q], mt, w.r[pos]);
        }
        g.sync();
    }
    double s = 0.0;
#pragma unroll 1
    for (int i = g.l; i < nL; i += G) s = fma(w.r[i], w.r[i], s);
    return g.sum(s);
}

// One FP64 refinement step of the LS solution by the corrected semi-normal
// equations: m += R^{-1} R^{-T} A^^T (e^ - A^ m), with the residual and
// A^^T r formed in FP64 from the FP64 values of A~ and R from the (FP32) QR.
template <class T, int G>
__device__ void refine(const WsT<typename T::TQ>& w, const SaiMat& A, int nL, int nS)
{
    const Grp<G> g;
    residual<T, G>(w, A, nL, nS, nullptr);  // r = A^ m - e^
#pragma unroll 1
    for (int t = g.l; t < nS; t += G) {
        const int32_t j = w.S[t];
        double gt = 0.0;
#pragma unroll 1
        for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
            const int pos = hfind<T::HL>(w.hk, w.hv, A.ri[q]);
            if (pos >= 0) gt = fma(-A.cv[q], w.r[pos], gt);
        }
        w.g[t] = gt;  // A^^T (e^ - A^ m)
    }
    g.sync();
    // R^T y = g (forward), R(t,i) = Q[i][t] for i > t
#pragma unroll 1
    for (int t = 0; t < nS; ++t) {
        const double yt = w.g[t] / (double)w.rd[t];
        g.sync();
        if (g.l == 0) w.g[t] = yt;
#pragma unroll 1
        for (int i = t + 1 + g.l; i < nS; i += G) w.g[i] = fma(-(double)w.Q[(size_t)i * T::LCAP + t], yt, w.g[i]);
        g.sync();
    }
    // R d = y (backward)
#pragma unroll 1
    for (int t = nS - 1; t >= 0; --t) {
        const double dt = w.g[t] / (double)w.rd[t];
        g.sync();
        if (g.l == 0) w.g[t] = dt;
#pragma unroll 1
        for (int i = g.l; i < t; i += G) w.g[i] = fma(-(double)w.Q[(size_t)t * T::LCAP + i], dt, w.g[i]);
        g.sync();
    }
#pragma unroll 1
    for (int t = g.l; t < nS; t += G) w.m[t] += w.g[t];
    g.sync();
}

// Algorithmic flops of one ls_update call that grows the factor of an
// nL x c block to nL x nS: the old reflectors on the new columns, the
// Householder factorisation of the trailing columns (each reflector applied
// to the later columns and to Q^T e), and the back substitution.
// (Integer arithmetic: the kernel's FP64 units are its bottleneck.)
__device__ __forceinline__ long long qr_flops(int nL, int c, int nS)
{
    const long long q = nS - c;
    long long f = 4 * q * ((long long)c * nL - (long long)c * (c - 1) / 2);
#pragma unroll 1
    for (int t = c; t < nS; ++t) f += 2LL * (nL - t) + 4LL * (nS - t) * (nL - t);
    return f + (long long)nS * nS;
}

// sum of nnz(A~(:,j)) over j in S (group-uniform result)
template <class T, int G>
__device__ int s_nnz(const WsT<typename T::TQ>& w, const SaiMat& A, int nS)
{
    const Grp<G> g;
    int c = 0;
#pragma unroll 1
    for (int t = g.l; t < nS; t += G) c += (int)(A.cp[w.S[t] + 1] - A.cp[w.S[t]]);
    return g.sum(c);
}

// fl: FP64 flops of the column; fq: flops of its QR (in the QR's type)
template <class T, int G>
__device__ int spai_column(const WsT<typename T::TQ>& w, const SaiMat& A, int32_t k, const SpaiArgs& a, int& nS_out,
                           int& l_out, double& rn_out, int& nL_out, long long& fl, long long& fq)
{
    const Grp<G> g;
    int nL, nS, nfact;
    col_init<T, G>(w, k, nL, nS, nfact);
    if (g.l == 0) w.S[0] = k;
    g.sync();
    int l = 0;
    double rn = 0.0;
    fl = 0;
    fq = 0;
#pragma unroll 1
    for (;;) {
        const int c0 = nfact;
        int st = ls_update<T, G>(w, A, nL, nS, nfact);
        if (st != ST_DONE) return st;
        const long long sn = s_nnz<T, G>(w, A, nS);
        fq += qr_flops(nL, c0, nS);
        if (sizeof(typename T::TQ) < sizeof(double)) {
            refine<T, G>(w, A, nL, nS);
            fl += 4 * sn + 2LL * nL + 2LL * nS * nS;
        }
        const double rn2 = residual<T, G>(w, A, nL, nS, nullptr);
        fl += 2 * sn + 2LL * nL;
        rn = sqrt(rn2);
        if (rn <= a.delta || l >= a.max_aug) break;
        // candidate set N \ S from the rows of L
#pragma unroll 1
        for (int q = g.l; q < T::HC; q += G) {
            w.ck[q] = -1;
            w.cf[q] = 0;
        }
        g.sync();
        bool ovf = false;
#pragma unroll 1
        for (int t = g.l; t < nS; t += G) {
            bool ins;
            int sl = hinsert<T::HC>(w.ck, w.S[t], ins);
            if (sl < 0) ovf = true;
            else w.cf[sl] = 1;
        }
        g.sync();
        int ncand = 0;
#pragma unroll 1
        for (int idx = g.l; idx < nL; idx += G) {
            const int32_t i = w.Lrow[idx];
#pragma unroll 1
            for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
                bool ins;
                int sl = hinsert<T::HC>(w.ck, A.rc[q], ins);
                if (sl < 0) ovf = true;
                ncand += ins;
            }
        }
        ncand = g.sum(ncand);
        if (g.any(ovf) || ncand + nS > T::HC / 2) return ST_OVERFLOW;
        g.sync();
        // compact the candidates (occupied slots not in S) to the front of ck,
        // in slot order, so that the scoring keeps every lane on a candidate;
        // a chunk is read whole before it is written, and the writes stay at
        // or below it
        int nc = 0;
#pragma unroll 1
        for (int s0 = 0; s0 < T::HC; s0 += G) {
            const int32_t j = w.ck[s0 + g.l];
            const bool keep = j >= 0 && !w.cf[s0 + g.l];
            const unsigned km = g.ballot(keep);
            if (keep) w.ck[nc + __popc(km & ((1u << g.l) - 1u))] = j;
            nc += __popc(km);
            g.sync();
        }
        // profitability keys and a per-lane sorted top list (the selection of
        // the mn smallest keys below does not depend on which lane scored what)
        unsigned long long top[MNMAX];
#pragma unroll
        for (int q = 0; q < MNMAX; ++q) top[q] = ULLONG_MAX;
        int fsc = 0;
        const double irn2 = 1.0 / rn2;  // rn2 > delta^2 >= 0 here
#pragma unroll 1
        for (int idx = g.l; idx < nc; idx += G) {
            const int32_t j = w.ck[idx];
            const double inj = A.icn[j];
            if (!(inj > 0.0)) continue;
            fsc += 2 * (int)(A.cp[j + 1] - A.cp[j]) + 5;  // r^T a_j, rho_j^2 and its key
            double d = 0.0;
#pragma unroll 1
            for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
                const int pos = hfind<T::HL>(w.hk, w.hv, A.ri[q]);
                if (pos >= 0) d = fma(w.r[pos], A.cv[q], d);
            }
            // rho_j^2 / ||r||^2 = 1 - (r^T a_j)^2 / (||a_j||^2 ||r||^2), in [0, 1]
            double tq = fma(-(d * d), inj * irn2, 1.0);
            tq = fmin(fmax(tq, 0.0), 1.0);
            unsigned long long x = (__double2ull_rz(tq * a.scale) << 32) | (unsigned)j;
#pragma unroll
            for (int q = 0; q < MNMAX; ++q) {
                const unsigned long long lo = top[q] < x ? top[q] : x;
                x = top[q] < x ? x : top[q];
                top[q] = lo;
            }
        }
        fl += g.sum(fsc);
        int added = 0;
#pragma unroll 1
        for (int sel = 0; sel < a.mn; ++sel) {
            const unsigned long long best = g.min_u64(top[0]);
            if (best == ULLONG_MAX) break;
            if (top[0] == best) {
#pragma unroll
                for (int q = 0; q < MNMAX - 1; ++q) top[q] = top[q + 1];
                top[MNMAX - 1] = ULLONG_MAX;
            }
            if (nS + added >= T::SCAP) return ST_OVERFLOW;
            if (g.l == 0) w.S[nS + added] = (int32_t)(best & 0xffffffffull);
            ++added;
        }
        g.sync();
        if (added == 0) break;
        nS += added;
        ++l;
    }
    nS_out = nS;
    l_out = l;
    rn_out = rn;
    nL_out = nL;
    return ST_DONE;
}

// PSAI(tol), reading (A): S^(l+1) = P(a^(l+1)) u S_kept^(l), a^(l+1) = |A~| a^(l).
template <class T, int G>
__device__ int psai_column(const WsT<typename T::TQ>& w, const SaiMat& A, int32_t k, const PsaiArgs& a, int& nS_out,
                           int& l_out, double& rn_pre, double& rn_post, int& nL_out, long long& fl, long long& fq)
{
    const Grp<G> g;
    int nL, nS, nfact;
    col_init<T, G>(w, k, nL, nS, nfact);
    if (g.l == 0) {
        w.S[0] = k;
        w.a0[0] = k;
    }
    g.sync();
    int na = 1;
    int32_t* apat = w.a0;
    int32_t* anew = w.a1;
    int l = 0;
    fl = 0;
    fq = 0;
#pragma unroll 1
    for (;;) {
        const int c0 = nfact;
        int st = ls_update<T, G>(w, A, nL, nS, nfact);
        if (st != ST_DONE) return st;
        const long long sn = s_nnz<T, G>(w, A, nS);
        fq += qr_flops(nL, c0, nS);
        if (sizeof(typename T::TQ) < sizeof(double)) {
            refine<T, G>(w, A, nL, nS);
            fl += 4 * sn + 2LL * nL + 2LL * nS * nS;
        }
        const double rn = sqrt(residual<T, G>(w, A, nL, nS, nullptr));
        fl += 2 * sn + 2LL * nL;
        double tolk = a.tol;
        if (a.tol_mode == 0) {
            int nz = 0;
#pragma unroll 1
            for (int t = g.l; t < nS; t += G) nz += (w.m[t] != 0.0);
            nz = g.sum(nz);
            tolk = (nz > 0 && A.norm1 > 0.0) ? a.delta / ((double)nz * A.norm1) : 0.0;
        }
        if (a.tol_mode == 2) {
            // PSAI(lfill): kp[t] = m_t is among the lfill largest in magnitude
            // (equal magnitudes to the smaller column index)
#pragma unroll 1
            for (int t = g.l; t < nS; t += G) {
                const double mt = fabs(w.m[t]);
                const int32_t jt = w.S[t];
                int rank = 0;
#pragma unroll 1
                for (int u = 0; u < nS; ++u) {
                    const double mu = fabs(w.m[u]);
                    rank += (mu > mt) || (mu == mt && w.S[u] < jt);
                }
                w.kp[t] = (uint8_t)(rank < a.lfill);
            }
        } else {
            // keep flags: kp[t] = |m_t| > tol_k
#pragma unroll 1
            for (int t = g.l; t < nS; t += G) w.kp[t] = (uint8_t)(fabs(w.m[t]) > tolk);
        }
        g.sync();
        if (rn <= a.delta || l >= a.lmax) {
            rn_pre = rn;
            rn_post = sqrt(residual<T, G>(w, A, nL, nS, w.kp));
            fl += 2 * sn + 2LL * nL;
            // compact the kept entries to the front of S / m (order preserved)
            int q = 0;
            if (g.l == 0) {
#pragma unroll 1
                for (int t = 0; t < nS; ++t)
                    if (w.kp[t]) {
                        w.S[q] = w.S[t];
                        w.m[q] = w.m[t];
                        ++q;
                    }
            }
            nS_out = g.bcast(q, 0);
            g.sync();
            l_out = l;
            nL_out = nL;
            return ST_DONE;
        }
        if (a.growth == 1) {
            // reading (C): S^(l+1) = S_kept^(l) u (P(a^(l+1)) \ P(a^(l))), so a
            // dropped position never comes back. Hash flags: 2 in P(a^(l)),
            // 8 kept member of S^(l), 4 in P(a^(l+1)).
#pragma unroll 1
            for (int q = g.l; q < T::HC; q += G) {
                w.ck[q] = -1;
                w.cf[q] = 0;
            }
            g.sync();
            bool ovf = false;
#pragma unroll 1
            for (int t = g.l; t < na; t += G) {
                bool ins;
                const int sl = hinsert<T::HC>(w.ck, apat[t], ins);
                if (sl < 0) ovf = true;
                else w.cf[sl] |= 2;
            }
            g.sync();
            int nk = 0;
#pragma unroll 1
            for (int t = g.l; t < nS; t += G) {
                if (!w.kp[t]) continue;
                ++nk;
                bool ins;
                const int sl = hinsert<T::HC>(w.ck, w.S[t], ins);
                if (sl < 0) ovf = true;
                else w.cf[sl] |= 8;
            }
            nk = g.sum(nk);
            g.sync();
#pragma unroll 1
            for (int t = 0; t < na; ++t) {
                const int32_t j = apat[t];
                const int64_t b = A.cp[j], e = A.cp[j + 1];
#pragma unroll 1
                for (int64_t q = b + g.l; q < e; q += G) {
                    bool ins;
                    const int sl = hinsert<T::HC>(w.ck, A.ri[q], ins);
                    if (sl < 0) ovf = true;
                    else w.cf[sl] |= 4;
                }
                g.sync();
            }
            if (g.any(ovf)) return ST_OVERFLOW;
            const unsigned lt = (1u << g.l) - 1u;
            int nb = 0, nf = 0;
#pragma unroll 1
            for (int s0 = 0; s0 < T::HC; s0 += G) {
                const int32_t key = w.ck[s0 + g.l];
                const uint8_t f = key >= 0 ? w.cf[s0 + g.l] : (uint8_t)0;
                const unsigned mn = g.ballot((f & 4) != 0);
                const unsigned mf = g.ballot((f & 4) != 0 && (f & 10) == 0);
                if (nb + __popc(mn) > T::SCAP) return ST_OVERFLOW;
                if (f & 4) anew[nb + __popc(mn & lt)] = key;
                nb += __popc(mn);
                nf += __popc(mf);
            }
            g.sync();
            if (nk + nf == 0) {
                // nothing kept and no new position: the column stops at loop l
                rn_pre = rn;
                rn_post = sqrt(residual<T, G>(w, A, nL, nS, w.kp));
                fl += 2 * sn + 2LL * nL;
                nS_out = 0;
                l_out = l;
                nL_out = nL;
                return ST_DONE;
            }
            if (nk + nf > T::SCAP) return ST_OVERFLOW;
            const bool dropped = nk < nS;
            if (dropped && g.l == 0) {  // the kept members, in list order, to the front
                int q = 0;
#pragma unroll 1
                for (int t = 0; t < nS; ++t)
                    if (w.kp[t]) w.S[q++] = w.S[t];
            }
            g.sync();
            int q = nk;
#pragma unroll 1
            for (int s0 = 0; s0 < T::HC; s0 += G) {  // then the frontier, in slot order
                const int32_t key = w.ck[s0 + g.l];
                const uint8_t f = key >= 0 ? w.cf[s0 + g.l] : (uint8_t)0;
                const bool fr = (f & 4) != 0 && (f & 10) == 0;
                const unsigned mf = g.ballot(fr);
                if (fr) w.S[q + __popc(mf & lt)] = key;
                q += __popc(mf);
            }
            g.sync();
            if (dropped) col_init<T, G>(w, k, nL, nS, nfact);  // refactor from scratch on the new pattern
            nS = q;
            int32_t* sw = apat;
            apat = anew;
            anew = sw;
            na = nb;
            ++l;
            continue;
        }
        // a^(l+1): union of the column patterns of a^(l); positions in entry order
#pragma unroll 1
        for (int q = g.l; q < T::HC; q += G) {
            w.ck[q] = -1;
            w.cf[q] = 0;
        }
        g.sync();
        int nb = 0;
#pragma unroll 1
        for (int t = 0; t < na; ++t) {
            const int32_t j = apat[t];
            const int64_t b = A.cp[j], e = A.cp[j + 1];
#pragma unroll 1
            for (int64_t base = b; base < e; base += G) {
                const int64_t q = base + g.l;
                bool isnew = false;
                int slot = 0;
                int32_t i = -1;
                if (q < e) {
                    i = A.ri[q];
                    slot = hinsert<T::HC>(w.ck, i, isnew);
                }
                if (g.any(slot < 0)) return ST_OVERFLOW;
                const unsigned mask = g.ballot(isnew);
                const int cnt = __popc(mask);
                if (nb + cnt > T::SCAP) return ST_OVERFLOW;
                if (isnew) anew[nb + __popc(mask & ((1u << g.l) - 1u))] = i;
                nb += cnt;
                g.sync();
            }
        }
        // cf = 1 marks members of S^(l) inside a^(l+1); a dropped member that is
        // not in a^(l+1) leaves the pattern (S shrinks)
        bool shrink = false;
#pragma unroll 1
        for (int t = g.l; t < nS; t += G) {
            const int sl = hslot<T::HC>(w.ck, w.S[t]);
            if (sl >= 0) w.cf[sl] = 1;
            else if (!w.kp[t]) shrink = true;
        }
        shrink = g.any(shrink);
        g.sync();
        if (!shrink) {
            // pure growth: append the members of a^(l+1) not in S, in list order
            int add = 0;
#pragma unroll 1
            for (int base = 0; base < nb; base += G) {
                const int t = base + g.l;
                bool fresh = false;
                int32_t j = -1;
                if (t < nb) {
                    j = anew[t];
                    fresh = w.cf[hslot<T::HC>(w.ck, j)] == 0;
                }
                const unsigned mask = g.ballot(fresh);
                if (nS + add + __popc(mask) > T::SCAP) return ST_OVERFLOW;
                if (fresh) w.S[nS + add + __popc(mask & ((1u << g.l) - 1u))] = j;
                add += __popc(mask);
            }
            g.sync();
            nS += add;
        } else {
            // rebuild from scratch with S = a^(l+1), then the kept members of
            // S^(l) outside a^(l+1)
            int q2 = nb;
            if (g.l == 0) {
#pragma unroll 1
                for (int t = 0; t < nS; ++t)
                    if (w.kp[t] && hslot<T::HC>(w.ck, w.S[t]) < 0) {
                        if (q2 < T::SCAP) apat[q2 - nb] = w.S[t];
                        ++q2;
                    }
            }
            q2 = g.bcast(q2, 0);
            g.sync();
            if (q2 > T::SCAP) return ST_OVERFLOW;
            // apat (old a^(l)) is free now: it holds the extra kept members
#pragma unroll 1
            for (int t = g.l; t < q2; t += G) w.S[t] = t < nb ? anew[t] : apat[t - nb];
            g.sync();
            col_init<T, G>(w, k, nL, nS, nfact);
            nS = q2;
        }
        // a^(l+1) becomes current
        int32_t* sw = apat;
        apat = anew;
        anew = sw;
        na = nb;
        ++l;
    }
}

// ---------------------------------------------------------------- lane tier
// The small tier with one lane per column: a warp builds 32 columns at once,
// each lane running its column's steps (the same steps as above) one after
// another, so a warp instruction serves 32 columns and no step needs a
// reduction across lanes. Each lane's workspace (|L| <= LT_L rows, |S| <=
// LT_S columns, the row and candidate hash tables) lives in shared memory,
// interleaved across the warp's lanes: element e of a lane's array sits at
// word e * 32 + lane, so the 32 lanes touch 32 different banks. A column
// that outgrows it is queued for tier 0, like the columns of the group form
// of the small tier.
constexpr int LT_L = 32, LT_S = 8, LT_HL = 64, LT_HC = 128;

// A lane's view of an array interleaved across the warp: element e at p[32 e].
template <class V>
struct LA {
    V* p;
    __device__ __forceinline__ V& operator[](int e) const { return p[(size_t)e * 32]; }
};

template <class TQ>
struct LaneLayout {
    // per-lane sizes in bytes of each array; each region holds 32 lanes
    static constexpr size_t Q = sizeof(TQ) * LT_L * LT_S, CV = sizeof(TQ) * LT_L, R = 8ull * LT_L, M = 8ull * LT_S,
                            G = 8ull * LT_S, BETA = sizeof(TQ) * LT_S, RD = sizeof(TQ) * LT_S, LROW = 4ull * LT_L,
                            HK = 4ull * LT_HL, HV = 1ull * LT_HL, S = 4ull * LT_S, A0 = 4ull * LT_S, A1 = 4ull * LT_S,
                            CK = 4ull * LT_HC, CF = 1ull * LT_HC, KP = 4ull * LT_S;
    static constexpr size_t OFF_Q = 0, OFF_CV = OFF_Q + 32 * Q, OFF_R = OFF_CV + 32 * CV, OFF_M = OFF_R + 32 * R,
                            OFF_G = OFF_M + 32 * M, OFF_BETA = OFF_G + 32 * G, OFF_RD = OFF_BETA + 32 * BETA,
                            OFF_LROW = OFF_RD + 32 * RD, OFF_HK = OFF_LROW + 32 * LROW, OFF_HV = OFF_HK + 32 * HK,
                            OFF_S = OFF_HV + 32 * HV, OFF_A0 = OFF_S + 32 * S, OFF_A1 = OFF_A0 + 32 * A0,
                            OFF_CK = OFF_A1 + 32 * A1, OFF_CF = OFF_CK + 32 * CK, OFF_KP = OFF_CF + 32 * CF;
    static constexpr size_t WARP_BYTES = OFF_KP + 32 * KP;  // one warp's 32 workspaces
};

template <class TQ>
struct LWs {
    LA<TQ> Q, cv, beta, rd;
    LA<double> r, m, g;
    LA<int32_t> Lrow, hk, S, a0, a1, ck;
    LA<uint8_t> hv, cf;  // row positions (< 32), candidate flags
    LA<int32_t> kp;
};

template <class TQ>
__device__ __forceinline__ LWs<TQ> bind_lane(char* wbase, int lane)
{
    using Lo = LaneLayout<TQ>;
    LWs<TQ> w;
    w.Q.p = (TQ*)(wbase + Lo::OFF_Q) + lane;
    w.cv.p = (TQ*)(wbase + Lo::OFF_CV) + lane;
    w.r.p = (double*)(wbase + Lo::OFF_R) + lane;
    w.m.p = (double*)(wbase + Lo::OFF_M) + lane;
    w.g.p = (double*)(wbase + Lo::OFF_G) + lane;
    w.beta.p = (TQ*)(wbase + Lo::OFF_BETA) + lane;
    w.rd.p = (TQ*)(wbase + Lo::OFF_RD) + lane;
    w.Lrow.p = (int32_t*)(wbase + Lo::OFF_LROW) + lane;
    w.hk.p = (int32_t*)(wbase + Lo::OFF_HK) + lane;
    w.hv.p = (uint8_t*)(wbase + Lo::OFF_HV) + lane;
    w.S.p = (int32_t*)(wbase + Lo::OFF_S) + lane;
    w.a0.p = (int32_t*)(wbase + Lo::OFF_A0) + lane;
    w.a1.p = (int32_t*)(wbase + Lo::OFF_A1) + lane;
    w.ck.p = (int32_t*)(wbase + Lo::OFF_CK) + lane;
    w.cf.p = (uint8_t*)(wbase + Lo::OFF_CF) + lane;
    w.kp.p = (int32_t*)(wbase + Lo::OFF_KP) + lane;
    return w;
}

// open-addressing tables of one lane (keys -1 = empty)
template <int H>
__device__ __forceinline__ int lh_find(const LA<int32_t>& hk, const LA<uint8_t>& hv, int32_t key)
{
    uint32_t s = hmix(key) & (H - 1);
#pragma unroll 1
    for (int probe = 0; probe < H; ++probe) {
        const int32_t k = hk[s];
        if (k == key) return hv[s];
        if (k == -1) return -1;
        s = (s + 1) & (H - 1);
    }
    return -1;
}

// slot of key, inserted if absent (ins set); -1 when the table is full
template <int H>
__device__ __forceinline__ int lh_insert(const LA<int32_t>& hk, int32_t key, bool& ins)
{
    uint32_t s = hmix(key) & (H - 1);
    ins = false;
#pragma unroll 1
    for (int probe = 0; probe < H; ++probe) {
        const int32_t k = hk[s];
        if (k == key) return (int)s;
        if (k == -1) {
            hk[s] = key;
            ins = true;
            return (int)s;
        }
        s = (s + 1) & (H - 1);
    }
    return -1;
}

template <int H>
__device__ __forceinline__ int lh_slot(const LA<int32_t>& hk, int32_t key)
{
    uint32_t s = hmix(key) & (H - 1);
#pragma unroll 1
    for (int probe = 0; probe < H; ++probe) {
        const int32_t k = hk[s];
        if (k == key) return (int)s;
        if (k == -1) return -1;
        s = (s + 1) & (H - 1);
    }
    return -1;
}

template <class TQ>
__device__ void lane_init(const LWs<TQ>& w, int32_t k, int& nL, int& nS, int& nfact)
{
#pragma unroll 1
    for (int q = 0; q < LT_HL; ++q) w.hk[q] = -1;
    bool ins;
    const int sl = lh_insert<LT_HL>(w.hk, k, ins);
    w.hv[sl] = 0;
    w.Lrow[0] = k;
    w.cv[0] = 1;
    nL = 1;
    nS = 1;
    nfact = 0;
}

// rows of column j of A~ into L, new rows at consecutive positions in entry order
template <class TQ>
__device__ bool lane_add_rows(const LWs<TQ>& w, const SaiMat& A, int32_t j, int& nL)
{
#pragma unroll 1
    for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
        const int32_t i = A.ri[q];
        bool ins;
        const int sl = lh_insert<LT_HL>(w.hk, i, ins);
        if (sl < 0) return false;
        if (ins) {
            if (nL >= LT_L) return false;
            w.hv[sl] = (uint8_t)nL;
            w.Lrow[nL] = i;
            ++nL;
        }
    }
    return true;
}

// the steps of ls_update for one lane: gather the new columns, old
// reflectors on them, Householder factorisation of the trailing block,
// back substitution
template <class TQ>
__device__ int lane_ls_update(const LWs<TQ>& w, const SaiMat& A, int& nL, int nS, int& nfact)
{
    const int nL_old = nL;
#pragma unroll 1
    for (int t = nfact; t < nS; ++t)
        if (!lane_add_rows(w, A, w.S[t], nL)) return ST_OVERFLOW;
#pragma unroll 1
    for (int t = 0; t < nS; ++t)
#pragma unroll 1
        for (int i = t < nfact ? nL_old : 0; i < nL; ++i) w.Q[t * LT_L + i] = 0;
#pragma unroll 1
    for (int i = nL_old; i < nL; ++i) w.cv[i] = 0;
#pragma unroll 1
    for (int t = nfact; t < nS; ++t) {
        const int32_t j = w.S[t];
#pragma unroll 1
        for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
            const int pos = lh_find<LT_HL>(w.hk, w.hv, A.ri[q]);
            if (pos >= 0) w.Q[t * LT_L + pos] = (TQ)A.cv[q];
        }
    }
#pragma unroll 1
    for (int jr = 0; jr < nfact; ++jr) {
        const TQ bj = w.beta[jr];
#pragma unroll 1
        for (int t = nfact; t < nS; ++t) {
            TQ d = 0;
#pragma unroll 1
            for (int i = jr; i < nL; ++i) d = fma(w.Q[jr * LT_L + i], w.Q[t * LT_L + i], d);
            const TQ f = bj * d;
#pragma unroll 1
            for (int i = jr; i < nL; ++i) w.Q[t * LT_L + i] = fma(-f, w.Q[jr * LT_L + i], w.Q[t * LT_L + i]);
        }
    }
#pragma unroll 1
    for (int t = nfact; t < nS; ++t) {
        TQ s2 = 0;
#pragma unroll 1
        for (int i = t; i < nL; ++i) s2 = fma(w.Q[t * LT_L + i], w.Q[t * LT_L + i], s2);
        if (!(s2 > (TQ)0)) return ST_SINGULAR;
        const TQ nrm = sqrt(s2);
        const TQ x0 = w.Q[t * LT_L + t];
        const TQ alpha = x0 >= (TQ)0 ? -nrm : nrm;
        const TQ bt = (TQ)1 / (nrm * (nrm + fabs(x0)));
        w.Q[t * LT_L + t] = x0 - alpha;
        w.rd[t] = alpha;
        w.beta[t] = bt;
#pragma unroll 1
        for (int t2 = t + 1; t2 <= nS; ++t2) {
            TQ d = 0;
            if (t2 < nS) {
#pragma unroll 1
                for (int i = t; i < nL; ++i) d = fma(w.Q[t * LT_L + i], w.Q[t2 * LT_L + i], d);
                const TQ f = bt * d;
#pragma unroll 1
                for (int i = t; i < nL; ++i) w.Q[t2 * LT_L + i] = fma(-f, w.Q[t * LT_L + i], w.Q[t2 * LT_L + i]);
            } else {
#pragma unroll 1
                for (int i = t; i < nL; ++i) d = fma(w.Q[t * LT_L + i], w.cv[i], d);
                const TQ f = bt * d;
#pragma unroll 1
                for (int i = t; i < nL; ++i) w.cv[i] = fma(-f, w.Q[t * LT_L + i], w.cv[i]);
            }
        }
    }
    nfact = nS;
#pragma unroll 1
    for (int i = 0; i < nS; ++i) w.m[i] = (double)w.cv[i];
#pragma unroll 1
    for (int t = nS - 1; t >= 0; --t) {
        const double mt = w.m[t] / (double)w.rd[t];
        w.m[t] = mt;
#pragma unroll 1
        for (int i = 0; i < t; ++i) w.m[i] = fma(-(double)w.Q[t * LT_L + i], mt, w.m[i]);
    }
    return ST_DONE;
}

template <class TQ>
__device__ double lane_residual(const LWs<TQ>& w, const SaiMat& A, int nL, int nS, bool use_kp)
{
#pragma unroll 1
    for (int i = 0; i < nL; ++i) w.r[i] = i == 0 ? -1.0 : 0.0;
#pragma unroll 1
    for (int t = 0; t < nS; ++t) {
        if (use_kp && !w.kp[t]) continue;
        const int32_t j = w.S[t];
        const double mt = w.m[t];
#pragma unroll 1
        for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
            const int pos = lh_find<LT_HL>(w.hk, w.hv, A.ri[q]);
            if (pos >= 0) w.r[pos] = fma(A.cv[q], mt, w.r[pos]);
        }
    }
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < nL; ++i) s = fma(w.r[i], w.r[i], s);
    return s;
}

template <class TQ>
__device__ void lane_refine(const LWs<TQ>& w, const SaiMat& A, int nL, int nS)
{
    lane_residual(w, A, nL, nS, false);
#pragma unroll 1
    for (int t = 0; t < nS; ++t) {
        const int32_t j = w.S[t];
        double gt = 0.0;
#pragma unroll 1
        for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
            const int pos = lh_find<LT_HL>(w.hk, w.hv, A.ri[q]);
            if (pos >= 0) gt = fma(-A.cv[q], w.r[pos], gt);
        }
        w.g[t] = gt;
    }
#pragma unroll 1
    for (int t = 0; t < nS; ++t) {
        const double yt = w.g[t] / (double)w.rd[t];
        w.g[t] = yt;
#pragma unroll 1
        for (int i = t + 1; i < nS; ++i) w.g[i] = fma(-(double)w.Q[i * LT_L + t], yt, w.g[i]);
    }
#pragma unroll 1
    for (int t = nS - 1; t >= 0; --t) {
        const double dt = w.g[t] / (double)w.rd[t];
        w.g[t] = dt;
#pragma unroll 1
        for (int i = 0; i < t; ++i) w.g[i] = fma(-(double)w.Q[t * LT_L + i], dt, w.g[i]);
    }
#pragma unroll 1
    for (int t = 0; t < nS; ++t) w.m[t] += w.g[t];
}

template <class TQ>
__device__ int lane_nnz(const LWs<TQ>& w, const SaiMat& A, int nS)
{
    int c = 0;
#pragma unroll 1
    for (int t = 0; t < nS; ++t) c += (int)(A.cp[w.S[t] + 1] - A.cp[w.S[t]]);
    return c;
}

template <class TQ>
__device__ int lane_spai(const LWs<TQ>& w, const SaiMat& A, int32_t k, const SpaiArgs& a, int& nS_out, int& l_out,
                         double& rn_out, int& nL_out, long long& fl, long long& fq)
{
    int nL, nS, nfact;
    lane_init(w, k, nL, nS, nfact);
    w.S[0] = k;
    int l = 0;
    double rn = 0.0;
    fl = 0;
    fq = 0;
#pragma unroll 1
    for (;;) {
        const int c0 = nfact;
        const int st = lane_ls_update(w, A, nL, nS, nfact);
        if (st != ST_DONE) return st;
        const long long sn = lane_nnz(w, A, nS);
        fq += qr_flops(nL, c0, nS);
        if (sizeof(TQ) < sizeof(double)) {
            lane_refine(w, A, nL, nS);
            fl += 4 * sn + 2LL * nL + 2LL * nS * nS;
        }
        const double rn2 = lane_residual(w, A, nL, nS, false);
        fl += 2 * sn + 2LL * nL;
        rn = sqrt(rn2);
        if (rn <= a.delta || l >= a.max_aug) break;
        // candidates N \ S from the rows of L (cf = 1 marks members of S)
#pragma unroll 1
        for (int q = 0; q < LT_HC; ++q) {
            w.ck[q] = -1;
            w.cf[q] = 0;
        }
#pragma unroll 1
        for (int t = 0; t < nS; ++t) {
            bool ins;
            const int sl = lh_insert<LT_HC>(w.ck, w.S[t], ins);
            if (sl < 0) return ST_OVERFLOW;
            w.cf[sl] = 1;
        }
        int ncand = 0;
#pragma unroll 1
        for (int idx = 0; idx < nL; ++idx) {
            const int32_t i = w.Lrow[idx];
#pragma unroll 1
            for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
                bool ins;
                if (lh_insert<LT_HC>(w.ck, A.rc[q], ins) < 0) return ST_OVERFLOW;
                ncand += ins;
            }
        }
        if (ncand + nS > LT_HC / 2) return ST_OVERFLOW;
        // keys of the candidates; the mn smallest in a sorted list
        unsigned long long top[MNMAX];
#pragma unroll
        for (int q = 0; q < MNMAX; ++q) top[q] = ULLONG_MAX;
        const double irn2 = 1.0 / rn2;
#pragma unroll 1
        for (int sl = 0; sl < LT_HC; ++sl) {
            const int32_t j = w.ck[sl];
            if (j < 0 || w.cf[sl]) continue;
            const double inj = A.icn[j];
            if (!(inj > 0.0)) continue;
            fl += 2 * (A.cp[j + 1] - A.cp[j]) + 5;
            double d = 0.0;
#pragma unroll 1
            for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
                const int pos = lh_find<LT_HL>(w.hk, w.hv, A.ri[q]);
                if (pos >= 0) d = fma(w.r[pos], A.cv[q], d);
            }
            double tq = fma(-(d * d), inj * irn2, 1.0);
            tq = fmin(fmax(tq, 0.0), 1.0);
            unsigned long long x = (__double2ull_rz(tq * a.scale) << 32) | (unsigned)j;
#pragma unroll
            for (int q = 0; q < MNMAX; ++q) {
                const unsigned long long lo = top[q] < x ? top[q] : x;
                x = top[q] < x ? x : top[q];
                top[q] = lo;
            }
        }
        int added = 0;
#pragma unroll
        for (int q = 0; q < MNMAX; ++q) {
            if (q >= a.mn || top[q] == ULLONG_MAX) break;
            if (nS + added >= LT_S) return ST_OVERFLOW;
            w.S[nS + added] = (int32_t)(top[q] & 0xffffffffull);
            ++added;
        }
        if (added == 0) break;
        nS += added;
        ++l;
    }
    nS_out = nS;
    l_out = l;
    rn_out = rn;
    nL_out = nL;
    return ST_DONE;
}

// PSAI(tol) for one lane: reading (A) growth, S^(l+1) = P(a^(l+1)) u S_kept^(l),
// and reading (C) (growth 1), as psai_column
template <class TQ>
__device__ int lane_psai(const LWs<TQ>& w, const SaiMat& A, int32_t k, const PsaiArgs& a, int& nS_out, int& l_out,
                         double& rn_pre, double& rn_post, int& nL_out, long long& fl, long long& fq)
{
    int nL, nS, nfact;
    lane_init(w, k, nL, nS, nfact);
    w.S[0] = k;
    w.a0[0] = k;
    int na = 1;
    bool cur0 = true;  // a^(l) in a0 (else a1)
    int l = 0;
    fl = 0;
    fq = 0;
#pragma unroll 1
    for (;;) {
        const LA<int32_t> apat = cur0 ? w.a0 : w.a1;
        const LA<int32_t> anew = cur0 ? w.a1 : w.a0;
        const int c0 = nfact;
        const int st = lane_ls_update(w, A, nL, nS, nfact);
        if (st != ST_DONE) return st;
        const long long sn = lane_nnz(w, A, nS);
        fq += qr_flops(nL, c0, nS);
        if (sizeof(TQ) < sizeof(double)) {
            lane_refine(w, A, nL, nS);
            fl += 4 * sn + 2LL * nL + 2LL * nS * nS;
        }
        const double rn = sqrt(lane_residual(w, A, nL, nS, false));
        fl += 2 * sn + 2LL * nL;
        double tolk = a.tol;
        if (a.tol_mode == 0) {
            int nz = 0;
#pragma unroll 1
            for (int t = 0; t < nS; ++t) nz += (w.m[t] != 0.0);
            tolk = (nz > 0 && A.norm1 > 0.0) ? a.delta / ((double)nz * A.norm1) : 0.0;
        }
        if (a.tol_mode == 2) {
#pragma unroll 1
            for (int t = 0; t < nS; ++t) {
                const double mt = fabs(w.m[t]);
                const int32_t jt = w.S[t];
                int rank = 0;
#pragma unroll 1
                for (int u = 0; u < nS; ++u) {
                    const double mu = fabs(w.m[u]);
                    rank += (mu > mt) || (mu == mt && w.S[u] < jt);
                }
                w.kp[t] = rank < a.lfill;
            }
        } else {
#pragma unroll 1
            for (int t = 0; t < nS; ++t) w.kp[t] = fabs(w.m[t]) > tolk;
        }
        if (rn <= a.delta || l >= a.lmax) {
            rn_pre = rn;
            rn_post = sqrt(lane_residual(w, A, nL, nS, true));
            fl += 2 * sn + 2LL * nL;
            int q = 0;
#pragma unroll 1
            for (int t = 0; t < nS; ++t)
                if (w.kp[t]) {
                    w.S[q] = w.S[t];
                    w.m[q] = w.m[t];
                    ++q;
                }
            nS_out = q;
            l_out = l;
            nL_out = nL;
            return ST_DONE;
        }
#pragma unroll 1
        for (int q = 0; q < LT_HC; ++q) {
            w.ck[q] = -1;
            w.cf[q] = 0;
        }
        if (a.growth == 1) {
            // reading (C): flags 2 in P(a^(l)), 8 kept member, 4 in P(a^(l+1))
#pragma unroll 1
            for (int t = 0; t < na; ++t) {
                bool ins;
                const int sl = lh_insert<LT_HC>(w.ck, apat[t], ins);
                if (sl < 0) return ST_OVERFLOW;
                w.cf[sl] = (uint8_t)(w.cf[sl] | 2);
            }
            int nk = 0;
#pragma unroll 1
            for (int t = 0; t < nS; ++t) {
                if (!w.kp[t]) continue;
                ++nk;
                bool ins;
                const int sl = lh_insert<LT_HC>(w.ck, w.S[t], ins);
                if (sl < 0) return ST_OVERFLOW;
                w.cf[sl] = (uint8_t)(w.cf[sl] | 8);
            }
#pragma unroll 1
            for (int t = 0; t < na; ++t) {
                const int32_t j = apat[t];
#pragma unroll 1
                for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
                    bool ins;
                    const int sl = lh_insert<LT_HC>(w.ck, A.ri[q], ins);
                    if (sl < 0) return ST_OVERFLOW;
                    w.cf[sl] = (uint8_t)(w.cf[sl] | 4);
                }
            }
            int nb = 0, nf = 0;
#pragma unroll 1
            for (int sl = 0; sl < LT_HC; ++sl) {
                const int32_t key = w.ck[sl];
                const int f = key >= 0 ? w.cf[sl] : 0;
                if (f & 4) {
                    if (nb >= LT_S) return ST_OVERFLOW;
                    anew[nb++] = key;
                    if ((f & 10) == 0) ++nf;
                }
            }
            if (nk + nf == 0) {
                rn_pre = rn;
                rn_post = sqrt(lane_residual(w, A, nL, nS, true));
                fl += 2 * sn + 2LL * nL;
                nS_out = 0;
                l_out = l;
                nL_out = nL;
                return ST_DONE;
            }
            if (nk + nf > LT_S) return ST_OVERFLOW;
            const bool dropped = nk < nS;
            if (dropped) {
                int q = 0;
#pragma unroll 1
                for (int t = 0; t < nS; ++t)
                    if (w.kp[t]) w.S[q++] = w.S[t];
            }
            int q = nk;
#pragma unroll 1
            for (int sl = 0; sl < LT_HC; ++sl) {
                const int32_t key = w.ck[sl];
                const int f = key >= 0 ? w.cf[sl] : 0;
                if ((f & 4) != 0 && (f & 10) == 0) w.S[q++] = key;
            }
            if (dropped) lane_init(w, k, nL, nS, nfact);
            nS = q;
            na = nb;
            cur0 = !cur0;
            ++l;
            continue;
        }
        // a^(l+1): the rows of the columns of a^(l), in entry order
        int nb = 0;
#pragma unroll 1
        for (int t = 0; t < na; ++t) {
            const int32_t j = apat[t];
#pragma unroll 1
            for (int64_t q = A.cp[j]; q < A.cp[j + 1]; ++q) {
                bool ins;
                const int32_t i = A.ri[q];
                const int sl = lh_insert<LT_HC>(w.ck, i, ins);
                if (sl < 0) return ST_OVERFLOW;
                if (ins) {
                    if (nb >= LT_S) return ST_OVERFLOW;
                    anew[nb++] = i;
                }
            }
        }
        bool shrink = false;
#pragma unroll 1
        for (int t = 0; t < nS; ++t) {
            const int sl = lh_slot<LT_HC>(w.ck, w.S[t]);
            if (sl >= 0) w.cf[sl] = 1;
            else if (!w.kp[t]) shrink = true;
        }
        if (!shrink) {
            int add = 0;
#pragma unroll 1
            for (int t = 0; t < nb; ++t) {
                const int32_t j = anew[t];
                if (w.cf[lh_slot<LT_HC>(w.ck, j)] == 0) {
                    if (nS + add >= LT_S) return ST_OVERFLOW;
                    w.S[nS + add] = j;
                    ++add;
                }
            }
            nS += add;
        } else {
            int q2 = nb;
#pragma unroll 1
            for (int t = 0; t < nS; ++t)
                if (w.kp[t] && lh_slot<LT_HC>(w.ck, w.S[t]) < 0) {
                    if (q2 >= LT_S) return ST_OVERFLOW;
                    apat[q2 - nb] = w.S[t];
                    ++q2;
                }
#pragma unroll 1
            for (int t = 0; t < q2; ++t) w.S[t] = t < nb ? anew[t] : apat[t - nb];
            lane_init(w, k, nL, nS, nfact);
            nS = q2;
        }
        na = nb;
        cur0 = !cur0;
        ++l;
    }
}

// Persistent lane-tier kernel: a warp takes 32 consecutive columns of the
// queue, one per lane, and takes the next 32 when all of its lanes are done.
template <class TQ, bool PSAI>
__global__ void __launch_bounds__(64) k_sai_lane(SaiMat A, SpaiArgs sa, PsaiArgs pa, const int32_t* __restrict__ work,
                                                  int32_t nwork, int* next, Out out, int32_t* ovf_list, int* ovf_cnt,
                                                  int* err, int tier_id)
{
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31;
    char* wbase = smem + (size_t)(threadIdx.x >> 5) * LaneLayout<TQ>::WARP_BYTES;
    const LWs<TQ> w = bind_lane<TQ>(wbase, lane);
    double work_bytes = 0.0;
    long long work_flops = 0, work_flops_q = 0;
#pragma unroll 1
    for (;;) {
        int first = 0;
        if (lane == 0) first = atomicAdd(next, 32);
        first = __shfl_sync(SAI_FULL, first, 0);
        if (first >= nwork) break;
        const int item = first + lane;
        if (item < nwork) {
            const int32_t k = work ? work[item] : item;
            int nS = 0, l = 0, nL = 0;
            double rn = 0.0, rpost = 0.0;
            long long cfl = 0, cfq = 0;
            int st = PSAI ? lane_psai(w, A, k, pa, nS, l, rn, rpost, nL, cfl, cfq)
                          : lane_spai(w, A, k, sa, nS, l, rn, nL, cfl, cfq);
            if (st == ST_DONE && nS > out.smax) st = ST_OVERFLOW;
            if (st == ST_DONE) {
                const size_t o = (size_t)k * out.smax;
                double cb = 0.0;
#pragma unroll 1
                for (int t = 0; t < nS; ++t) {
                    out.rows[o + t] = w.S[t];
                    out.vals[o + t] = w.m[t];
                    cb += 12.0 * (double)(A.cp[w.S[t] + 1] - A.cp[w.S[t]]) + 12.0;
                }
#pragma unroll 1
                for (int t = 0; t < nL; ++t) cb += 4.0 * (double)(A.rp[w.Lrow[t] + 1] - A.rp[w.Lrow[t]]);
                work_bytes += cb;
                work_flops += cfl;
                work_flops_q += cfq;
                out.cnt[k] = nS;
                out.loops[k] = l;
                out.res[k] = rn;
                if (out.res_post) out.res_post[k] = rpost;
                out.tier[k] = tier_id;
            } else if (st == ST_OVERFLOW) {
                if (ovf_list) ovf_list[atomicAdd(ovf_cnt, 1)] = k;
                else atomicOr(err, 1);
            } else {
                atomicOr(err, 2);
            }
        }
        __syncwarp();
    }
    work_bytes = warp_sum(work_bytes);
    const double wf = warp_sum((double)work_flops), wq = warp_sum((double)work_flops_q);
    if (lane == 0 && work_bytes > 0.0) {
        const bool q32 = sizeof(TQ) < sizeof(double);
        atomicAdd(&d_swork[2 * PROF_SAI_BUILD], work_bytes);
        atomicAdd(&d_swork[2 * PROF_SAI_BUILD + 1], wf + (q32 ? 0.0 : wq));
        if (q32) atomicAdd(&d_swork32, wq);
    }
}

// Persistent build kernel: each warp takes 32/G consecutive columns from the
// atomic queue (work list, or 0..nwork-1), one per group of G lanes, until
// the queue is empty. The groups of a warp start their columns together and
// wait for one another before the next ones, so that columns of similar
// shape run their steps in the same instructions rather than one group after
// another. SMEM: the workspaces live in dynamic shared memory, one per
// group; otherwise in gscratch, one per group of the grid.
template <class T, int G, bool SMEM, bool PSAI>
__global__ void __launch_bounds__(256) k_sai(SaiMat A, SpaiArgs sa, PsaiArgs pa, const int32_t* __restrict__ work,
                                             int32_t nwork, int* next, char* gscratch, Out out, int32_t* ovf_list,
                                             int* ovf_cnt, int* err, int tier_id)
{
    extern __shared__ __align__(16) char smem[];
    const Grp<G> g;
    constexpr int GPW = 32 / G;  // groups per warp
    const int grp = (int)(threadIdx.x >> 5) * GPW + (g.base / G);  // group index within the block
    char* base = SMEM ? smem + (size_t)grp * T::STRIDE
                      : gscratch + ((size_t)blockIdx.x * (blockDim.x / G) + grp) * T::STRIDE;
    const WsT<typename T::TQ> w = bind_ws<T>(base);
    double work_bytes = 0.0;
    long long work_flops = 0, work_flops_q = 0;
#pragma unroll 1
    for (;;) {
        int first = 0;
        if ((threadIdx.x & 31) == 0) first = atomicAdd(next, GPW);
        first = __shfl_sync(SAI_FULL, first, 0);
        if (first >= nwork) break;
        const int item = first + g.base / G;
        if (item < nwork) {
            const int32_t k = work ? work[item] : item;
            int nS = 0, l = 0, nL = 0;
            double rn = 0.0, rpost = 0.0;
            long long cfl = 0, cfq = 0;
            int st = PSAI ? psai_column<T, G>(w, A, k, pa, nS, l, rn, rpost, nL, cfl, cfq)
                          : spai_column<T, G>(w, A, k, sa, nS, l, rn, nL, cfl, cfq);
            const bool big = out.big_smax > 0;
            if (st == ST_DONE) {
                if (nS > (big ? out.big_smax : out.smax)) st = ST_OVERFLOW;
            }
            if (st == ST_DONE) {
                int32_t* orow = big ? out.big_rows + (size_t)item * out.big_smax : out.rows + (size_t)k * out.smax;
                double* oval = big ? out.big_vals + (size_t)item * out.big_smax : out.vals + (size_t)k * out.smax;
#pragma unroll 1
                for (int t = g.l; t < nS; t += G) {
                    orow[t] = w.S[t];
                    oval[t] = w.m[t];
                }
                if (big && g.l == 0) out.big_slot[k] = item;
                double cb = 0.0;
#pragma unroll 1
                for (int t = g.l; t < nS; t += G) cb += 12.0 * (double)(A.cp[w.S[t] + 1] - A.cp[w.S[t]]) + 12.0;
#pragma unroll 1
                for (int t = g.l; t < nL; t += G) cb += 4.0 * (double)(A.rp[w.Lrow[t] + 1] - A.rp[w.Lrow[t]]);
                work_bytes += g.sum(cb);
                work_flops += cfl;
                work_flops_q += cfq;
                if (g.l == 0) {
                    out.cnt[k] = nS;
                    out.loops[k] = l;
                    out.res[k] = rn;
                    if (out.res_post) out.res_post[k] = rpost;
                    out.tier[k] = tier_id;
                }
            } else if (st == ST_OVERFLOW) {
                if (g.l == 0) {
                    if (ovf_list) {
                        int p = atomicAdd(ovf_cnt, 1);
                        ovf_list[p] = k;
                    } else {
                        atomicOr(err, 1);
                    }
                }
            } else {
                if (g.l == 0) atomicOr(err, 2);
            }
        }
        __syncwarp();
    }
    if (g.l == 0 && work_bytes > 0.0) {
        const bool q32 = sizeof(typename T::TQ) < sizeof(double);
        atomicAdd(&d_swork[2 * PROF_SAI_BUILD], work_bytes);
        atomicAdd(&d_swork[2 * PROF_SAI_BUILD + 1], (double)(work_flops + (q32 ? 0 : work_flops_q)));
        if (q32) atomicAdd(&d_swork32, (double)work_flops_q);
    }
}

// One warp per column: rank-sort the column's slots by row into CSC (the
// large tier's columns from their own slots).
__global__ void k_assemble(int32_t n, int32_t smax, const int32_t* cnt, const int32_t* rows, const double* vals,
                           const int64_t* cp, int32_t* ri, double* v, const int32_t* big_slot, int32_t big_smax,
                           const int32_t* big_rows, const double* big_vals)
{
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= n) return;
    const int c = cnt[k];
    const int bs = big_slot ? big_slot[k] : -1;
    const int32_t* rk = bs >= 0 ? big_rows + (size_t)bs * big_smax : rows + (size_t)k * smax;
    const double* vk = bs >= 0 ? big_vals + (size_t)bs * big_smax : vals + (size_t)k * smax;
#pragma unroll 1
    for (int t = lane; t < c; t += 32) {
        const int32_t r = rk[t];
        int rank = 0;
#pragma unroll 1
        for (int u = 0; u < c; ++u) rank += rk[u] < r;
        ri[cp[k] + rank] = r;
        v[cp[k] + rank] = vk[t];
    }
}

__global__ void k_stats(int32_t n, const int32_t* loops, const double* res, double delta, int* out)
{
    int nc = 0, lm = 0;
#pragma unroll 1
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        nc += res[k] > delta;
        lm = max(lm, loops[k]);
    }
    nc = warp_sum_int(nc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = max(lm, __shfl_xor_sync(SAI_FULL, lm, o));
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], nc);
        atomicMax(&out[1], lm);
    }
}

// columns not built in this call (outside a column list) hold tier -1
__global__ void k_tier_count(int32_t n, const int32_t* tier, int* out)
{
    int c[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int t = tier[k];
#pragma unroll
        for (int q = 0; q < 6; ++q) c[q] += t == q;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int w = warp_sum_int(c[q]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&out[2 + q], w);
    }
}

// icn[j] = 1/cn2[j] (0 where cn2[j] = 0: an empty column scores no key)
__global__ void k_recip(int32_t n, const double* __restrict__ cn2, double* __restrict__ icn)
{
#pragma unroll 1
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        icn[j] = cn2[j] > 0.0 ? 1.0 / cn2[j] : 0.0;
}

int g_num_sms = 0;

// Launches one tier of the build over a work list: G lanes per column,
// workspaces in shared memory (SMEM: as many blocks per SM as fit) or in a
// pool buffer (blocks_per_sm_t12 blocks of 8 warps per SM, no more than the
// list needs).
template <class T, int G, bool SMEM, bool PSAI>
sai_status launch_tier(const SaiMat& A, const SpaiArgs& sa, const PsaiArgs& pa, const int32_t* work, int32_t nwork,
                       int* next, const Out& out, int32_t* ovf_list, int* ovf_cnt, int* err, int tier_id,
                       const sai_build_config& cfg, cudaStream_t st)
{
    if (nwork <= 0) return SAI_OK;
    const int warps_per_block = SMEM ? cfg.warps_t0 : 8;
    const int threads = 32 * warps_per_block;
    const int groups = threads / G;
    int blocks;
    Buf scratch;
    size_t smem = 0;
    if (SMEM) {
        smem = T::STRIDE * groups;
        SAI_CUDA(cudaFuncSetAttribute(k_sai<T, G, SMEM, PSAI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sai<T, G, SMEM, PSAI>, threads, smem));
        if (per_sm < 1) per_sm = 1;
        blocks = g_num_sms * per_sm;
    } else {
        blocks = g_num_sms * cfg.blocks_per_sm_t12;
        const int need = (nwork + groups - 1) / groups;
        if (blocks > need) blocks = need;
        SAI_TRY(scratch.alloc(T::STRIDE * (size_t)groups * blocks, st, true));
    }
    SAI_CUDA(cudaMemsetAsync(next, 0, sizeof(int), st));
    {
        ProfScope ps(PROF_SAI_BUILD, st);
        k_sai<T, G, SMEM, PSAI><<<SAI_GRID(blocks), threads, smem, st>>>(A, sa, pa, work, nwork, next,
                                                                        scratch.as<char>(), out, ovf_list, ovf_cnt,
                                                                        err, tier_id);
    }
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

// The lane form of the small tier: one warp per block (its 32 workspaces
// take the block's shared memory), as many blocks as fit on each SM, no more
// than the list needs.
template <class TQ, bool PSAI>
sai_status launch_lane(const SaiMat& A, const SpaiArgs& sa, const PsaiArgs& pa, const int32_t* work, int32_t nwork,
                       int* next, const Out& out, int32_t* ovf_list, int* ovf_cnt, int* err, cudaStream_t st)
{
    if (nwork <= 0) return SAI_OK;
    const size_t smem = LaneLayout<TQ>::WARP_BYTES;
    SAI_CUDA(cudaFuncSetAttribute(k_sai_lane<TQ, PSAI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SAI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sai_lane<TQ, PSAI>, 32, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)g_num_sms * per_sm;
    const int64_t need = ((int64_t)nwork + 31) / 32;
    if (blocks > need) blocks = need;
    SAI_CUDA(cudaMemsetAsync(next, 0, sizeof(int), st));
    {
        ProfScope ps(PROF_SAI_BUILD, st);
        k_sai_lane<TQ, PSAI><<<SAI_GRID(blocks), 32, smem, st>>>(A, sa, pa, work, nwork, next, out, ovf_list, ovf_cnt,
                                                                 err, 4);
    }
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

// The large-pattern tier: one warp per column and per block, as many as
// the list needs up to one per SM, fewer when their workspaces (~68 MB
// each in FP64) would take more than a quarter of the free device memory
// (16 GB at most); the columns write to slots of their own.
template <class T, bool PSAI>
sai_status launch_big(const SaiMat& A, const SpaiArgs& sa, const PsaiArgs& pa, const int32_t* work, int32_t nwork,
                      int* next, Out out, int* err, cudaStream_t st, Buf& big_rows, Buf& big_vals)
{
    if (nwork <= 0) return SAI_OK;
    size_t fr = 0, tot = 0;
    SAI_CUDA(cudaMemGetInfo(&fr, &tot));
    size_t budget = fr / 4;
    if (budget > (size_t(16) << 30)) budget = size_t(16) << 30;
    int64_t warps = nwork < g_num_sms ? nwork : g_num_sms;
    const int64_t fit = (int64_t)(budget / T::STRIDE);
    if (warps > fit) warps = fit > 0 ? fit : 1;
    Buf scratch;
    SAI_TRY(scratch.alloc(T::STRIDE * (size_t)warps, st, true));
    SAI_TRY(big_rows.alloc(sizeof(int32_t) * (size_t)nwork * T::SCAP, st, true));
    SAI_TRY(big_vals.alloc(sizeof(double) * (size_t)nwork * T::SCAP, st, true));
    out.big_smax = T::SCAP;
    out.big_rows = big_rows.as<int32_t>();
    out.big_vals = big_vals.as<double>();
    SAI_CUDA(cudaMemsetAsync(next, 0, sizeof(int), st));
    {
        ProfScope ps(PROF_SAI_BUILD, st);
        k_sai<T, 32, false, PSAI><<<SAI_GRID(warps), 32, 0, st>>>(A, sa, pa, work, nwork, next, scratch.as<char>(), out,
                                                                  nullptr, nullptr, err, 5);
    }
    SAI_CUDA(cudaGetLastError());
    return SAI_OK;
}

template <class TQ>
struct Tiers;
template <>
struct Tiers<double> {
    using TS = TierS;
    using T0 = Tier0;
    using T1 = Tier1;
    using T2 = Tier2;
    using T3 = Tier3;
    using T4 = Tier4;
};
template <>
struct Tiers<float> {
    using TS = TierSF;
    using T0 = Tier0F;
    using T1 = Tier1F;
    using T2 = Tier2F;
    using T3 = Tier3F;
    using T4 = Tier4F;
};

// Build configuration: the warps per block of the shared-memory tiers, the
// blocks per SM of the global-memory tiers, the order of the first tier's
// work queue (heavy_first: the columns of A~ with more than twice the
// average number of entries, in index order, then the rest, in index order)
// and the first tier (0: tier 0; 1 or 2: the small tier with 8- or 16-lane
// groups; 3: its lane form). Only first_tier changes a column's arithmetic
// (its group size); the rest changes the schedule alone. SPAI and PSAI keep
// a configuration each (their columns' shapes differ).
std::mutex g_cfg_mu;
sai_build_config g_cfg[2] = {{8, 2, 0, 0, 0.f}, {8, 2, 0, 0, 0.f}};

sai_build_config current_config(bool psai)
{
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    return g_cfg[psai ? 1 : 0];
}

// heavy[i] = nnz(A~ e_{list_i}) > thr (list = nullptr: i itself)
__global__ void k_heavy_flags(int32_t m, const int32_t* __restrict__ list, const int64_t* __restrict__ cp, double thr,
                              int32_t* __restrict__ flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = list ? list[i] : (int32_t)i;
        flag[i] = (double)(cp[k + 1] - cp[k]) > thr;
    }
}

// stable partition: heavy entries first (pos = prefix of heavy flags), then
// the others (pos = H + i - prefix)
__global__ void k_heavy_scatter(int32_t m, const int32_t* __restrict__ list, const int32_t* __restrict__ flag,
                                const int64_t* __restrict__ pre, int32_t* __restrict__ out)
{
    const int64_t H = pre[m];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = list ? list[i] : (int32_t)i;
        out[flag[i] ? pre[i] : H + (i - pre[i])] = k;
    }
}

template <bool PSAI, class TQ>
sai_status build_common(const sai_split_s* h, const SpaiArgs& sa, const PsaiArgs& pa, int32_t smax, double delta,
                        cudaStream_t st, bool async, sai_precond_s* P, const int32_t* cols = nullptr,
                        int32_t ncols = -1, const sai_build_config* cfgp = nullptr)
{
    const sai_build_config cfg = cfgp ? *cfgp : current_config(PSAI);
    if (g_num_sms == 0) {
        int dev = 0;
        SAI_CUDA(cudaGetDevice(&dev));
        SAI_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int32_t n = h->n;
    P->n = n;
    cudaEvent_t e0, e1;
    SAI_CUDA(cudaEventCreate(&e0));
    SAI_CUDA(cudaEventCreate(&e1));
    SAI_CUDA(cudaEventRecord(e0, st));
    SaiMat A;
    A.n = n;
    A.cp = h->At_cp.as<int64_t>();
    A.ri = h->At_ri.as<int32_t>();
    A.cv = h->At_v.as<double>();
    A.rp = h->Atr_rp.as<int64_t>();
    A.rc = h->Atr_ci.as<int32_t>();
    A.norm1 = h->norm1;

    const size_t nn = (size_t)(n > 0 ? n : 1);
    Buf icn;
    SAI_TRY(icn.alloc(sizeof(double) * nn, st, true));
    if (n > 0) {
        const unsigned gi = sai_div_up(n, 256) < (unsigned)g_num_sms * 8 ? sai_div_up(n, 256) : g_num_sms * 8;
        k_recip<<<SAI_GRID(gi), 256, 0, st>>>(n, h->colnorm2.as<double>(), icn.as<double>());
        SAI_CUDA(cudaGetLastError());
    }
    A.icn = icn.as<double>();
    Buf cnt, rows, vals, tier, ctr, ovf0, ovf1, ovfs, bslot, brows, bvals;
    bool big_used = false;
    SAI_TRY(cnt.alloc(sizeof(int32_t) * nn, st, true));
    SAI_TRY(rows.alloc(sizeof(int32_t) * nn * smax, st, true));
    SAI_TRY(vals.alloc(sizeof(double) * nn * smax, st, true));
    SAI_TRY(tier.alloc(sizeof(int32_t) * nn, st, true));
    SAI_TRY(P->loops.alloc(sizeof(int32_t) * nn, st, async));
    SAI_TRY(P->res.alloc(sizeof(double) * nn, st, async));
    SAI_TRY(P->res_post.alloc(sizeof(double) * nn, st, async));
    SAI_TRY(ctr.alloc(sizeof(int) * 16, st, true));
    SAI_TRY(ovf0.alloc(sizeof(int32_t) * nn, st, true));
    SAI_TRY(ovf1.alloc(sizeof(int32_t) * nn, st, true));
    if (cfg.first_tier != 0) SAI_TRY(ovfs.alloc(sizeof(int32_t) * nn, st, true));
    SAI_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(int) * 16, st));
    SAI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * nn, st));
    SAI_CUDA(cudaMemsetAsync(P->res_post.p, 0, sizeof(double) * nn, st));
    // per-column outputs start defined: a column list builds only some columns
    SAI_CUDA(cudaMemsetAsync(tier.p, 0xff, sizeof(int32_t) * nn, st));
    SAI_CUDA(cudaMemsetAsync(P->loops.p, 0, sizeof(int32_t) * nn, st));
    SAI_CUDA(cudaMemsetAsync(P->res.p, 0, sizeof(double) * nn, st));
    // [0] next, [1..2] ovf counts t0, t1, [3] err, [4..11] stats (n_c, l_m, columns per tier), [12] ovf
    // count t2, [13] ovf count of the small tier, [14] ovf count t3
    int* c = ctr.as<int>();
    Out out;
    out.smax = smax;
    out.cnt = cnt.as<int32_t>();
    out.rows = rows.as<int32_t>();
    out.vals = vals.as<double>();
    out.loops = P->loops.as<int32_t>();
    out.res = P->res.as<double>();
    out.res_post = PSAI ? P->res_post.as<double>() : nullptr;
    out.tier = tier.as<int32_t>();
    SAI_TRY(bslot.alloc(sizeof(int32_t) * nn, st, true));
    out.big_smax = 0;
    out.big_slot = bslot.as<int32_t>();
    out.big_rows = nullptr;
    out.big_vals = nullptr;

    using TS = typename Tiers<TQ>::TS;
    using T0 = typename Tiers<TQ>::T0;
    using T1 = typename Tiers<TQ>::T1;
    using T2 = typename Tiers<TQ>::T2;
    using T3 = typename Tiers<TQ>::T3;
    using T4 = typename Tiers<TQ>::T4;
    // tier-0 work queue: all columns (or the given list), optionally heavy ones first
    const int32_t nq = cols ? ncols : n;
    const int32_t* queue = cols;
    Buf qbuf, qflag, qpre;
    if (cfg.heavy_first && nq > 0) {
        SAI_TRY(qbuf.alloc(sizeof(int32_t) * (size_t)nq, st, true));
        SAI_TRY(qflag.alloc(sizeof(int32_t) * (size_t)nq, st, true));
        SAI_TRY(qpre.alloc(sizeof(int64_t) * ((size_t)nq + 1), st, true));
        const double thr = n > 0 ? 2.0 * (double)h->nnz_At / (double)n : 0.0;
        const unsigned g = sai_div_up(nq, 256) < (unsigned)g_num_sms * 8 ? sai_div_up(nq, 256) : g_num_sms * 8;
        k_heavy_flags<<<SAI_GRID(g), 256, 0, st>>>(nq, cols, A.cp, thr, qflag.as<int32_t>());
        SAI_TRY(sai_scan_counts_i32(qflag.as<int32_t>(), qpre.as<int64_t>(), nq, st));
        k_heavy_scatter<<<SAI_GRID(g), 256, 0, st>>>(nq, cols, qflag.as<int32_t>(), qpre.as<int64_t>(),
                                                     qbuf.as<int32_t>());
        SAI_CUDA(cudaGetLastError());
        queue = qbuf.as<int32_t>();
    }
    // the small tier first (first_tier 1 or 2): its overflows are tier 0's queue
    const int32_t* q0 = queue;
    int32_t n0 = nq;
    if (cfg.first_tier != 0) {
        if (cfg.first_tier == 3)
            SAI_TRY((launch_lane<TQ, PSAI>(A, sa, pa, queue, nq, c + 0, out, ovfs.as<int32_t>(), c + 13, c + 3, st)));
        else if (cfg.first_tier == 1)
            SAI_TRY((launch_tier<TS, 8, true, PSAI>(A, sa, pa, queue, nq, c + 0, out, ovfs.as<int32_t>(), c + 13,
                                                    c + 3, 4, cfg, st)));
        else
            SAI_TRY((launch_tier<TS, 16, true, PSAI>(A, sa, pa, queue, nq, c + 0, out, ovfs.as<int32_t>(), c + 13,
                                                     c + 3, 4, cfg, st)));
        SAI_CUDA(cudaMemcpyAsync(&n0, c + 13, sizeof(int), cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        q0 = ovfs.as<int32_t>();
    }
    SAI_TRY((launch_tier<T0, 32, true, PSAI>(A, sa, pa, q0, n0, c + 0, out, ovf0.as<int32_t>(), c + 1, c + 3, 0, cfg,
                                             st)));
    int hc[4];
    SAI_CUDA(cudaMemcpyAsync(hc, c, sizeof(hc), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    if (hc[1] > 0) {
        SAI_TRY((launch_tier<T1, 32, false, PSAI>(A, sa, pa, ovf0.as<int32_t>(), hc[1], c + 0, out,
                                                     ovf1.as<int32_t>(), c + 2, c + 3, 1, cfg, st)));
        SAI_CUDA(cudaMemcpyAsync(hc, c, sizeof(hc), cudaMemcpyDeviceToHost, st));
        SAI_CUDA(cudaStreamSynchronize(st));
        if (hc[2] > 0) {
            // tier 2 queues its overflows in ovf0 (tier 1's input, no longer read)
            SAI_TRY((launch_tier<T2, 32, false, PSAI>(A, sa, pa, ovf1.as<int32_t>(), hc[2], c + 0, out,
                                                         ovf0.as<int32_t>(), c + 12, c + 3, 2, cfg, st)));
            int h3 = 0;
            SAI_CUDA(cudaMemcpyAsync(&h3, c + 12, sizeof(int), cudaMemcpyDeviceToHost, st));
            SAI_CUDA(cudaStreamSynchronize(st));
            if (h3 > 0) {
                // tier 3 queues its overflows in ovf1 (tier 2's input, no longer read)
                SAI_TRY((launch_tier<T3, 32, false, PSAI>(A, sa, pa, ovf0.as<int32_t>(), h3, c + 0, out,
                                                             ovf1.as<int32_t>(), c + 14, c + 3, 3, cfg, st)));
                int h4 = 0;
                SAI_CUDA(cudaMemcpyAsync(&h4, c + 14, sizeof(int), cudaMemcpyDeviceToHost, st));
                SAI_CUDA(cudaStreamSynchronize(st));
                if (h4 > 0) {
                    SAI_CUDA(cudaMemsetAsync(bslot.p, 0xff, sizeof(int32_t) * nn, st));
                    big_used = true;
                    SAI_TRY((launch_big<T4, PSAI>(A, sa, pa, ovf1.as<int32_t>(), h4, c + 0, out, c + 3, st, brows,
                                                  bvals)));
                }
            }
        }
    }
    // assemble M (CSC, rows ascending) and its CSR copy
    SAI_TRY(P->M_cp.alloc(sizeof(int64_t) * (nn + 1), st, async));
    SAI_TRY(sai_scan_counts_i32(cnt.as<int32_t>(), P->M_cp.as<int64_t>(), n, st));
    int64_t nnzM = 0;
    SAI_CUDA(cudaMemcpyAsync(&nnzM, P->M_cp.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaMemcpyAsync(hc, c, sizeof(hc), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    if (hc[3] & 2) return SAI_SINGULAR;
    if (hc[3] & 1) return SAI_PATTERN_OVERFLOW;
    P->nnz = nnzM;
    SAI_TRY(P->M_ri.alloc(sizeof(int32_t) * (size_t)(nnzM > 0 ? nnzM : 1), st, async));
    SAI_TRY(P->M_v.alloc(sizeof(double) * (size_t)(nnzM > 0 ? nnzM : 1), st, async));
    if (n > 0)
        k_assemble<<<SAI_GRID(sai_div_up((int64_t)n * 32, 256)), 256, 0, st>>>(
            n, smax, cnt.as<int32_t>(), rows.as<int32_t>(), vals.as<double>(), P->M_cp.as<int64_t>(),
            P->M_ri.as<int32_t>(), P->M_v.as<double>(), big_used ? bslot.as<int32_t>() : nullptr, T4::SCAP,
            big_used ? brows.as<int32_t>() : nullptr, big_used ? bvals.as<double>() : nullptr);
    SAI_CUDA(cudaGetLastError());
    SAI_TRY(sai_csc_to_csr(n, n, nnzM, P->M_cp.as<int64_t>(), P->M_ri.as<int32_t>(), P->M_v.as<double>(), P->Mr_rp,
                           P->Mr_ci, P->Mr_v, st, async));
    SAI_CUDA(cudaEventRecord(e1, st));
    if (n > 0) {
        k_stats<<<SAI_GRID(g_num_sms * 2), 256, 0, st>>>(n, P->loops.as<int32_t>(), P->res.as<double>(), delta, c + 4);
        k_tier_count<<<SAI_GRID(g_num_sms * 2), 256, 0, st>>>(n, tier.as<int32_t>(), c + 4);
    }
    SAI_CUDA(cudaGetLastError());
    int hs[8];
    SAI_CUDA(cudaMemcpyAsync(hs, c + 4, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SAI_CUDA(cudaStreamSynchronize(st));
    P->n_c = hs[0];
    P->l_m = hs[1];
    for (int q = 0; q < 6; ++q) P->n_tier[q] = hs[2 + q];
    SAI_CUDA(cudaEventElapsedTime(&P->ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SAI_OK;
}

}  // namespace

sai_status sai_spai_build(const sai_split_s* h, const sai_spai_params* prm, cudaStream_t st, bool async,
                          sai_precond_s* P)
{
    if (!h || !prm || !P) return SAI_INVALID_ARG;
    if (prm->mn < 1 || prm->mn > MNMAX || prm->max_aug < 0 || prm->key_bits < 1 || prm->key_bits > 31 ||
        !(prm->delta >= 0.0))
        return SAI_INVALID_ARG;
    if (prm->precision != SAI_FP64 && prm->precision != SAI_FP32_REFINE64) return SAI_INVALID_ARG;
    SpaiArgs sa;
    sa.delta = prm->delta;
    sa.scale = ldexp(1.0, prm->key_bits);
    sa.mn = prm->mn;
    sa.max_aug = prm->max_aug;
    PsaiArgs pa = {};
    long long bound = 1 + (long long)prm->mn * prm->max_aug;
    int32_t smax = (int32_t)(bound < Tier2::SCAP ? bound : Tier2::SCAP);
    if (prm->precision == SAI_FP32_REFINE64) return build_common<false, float>(h, sa, pa, smax, prm->delta, st, async, P);
    return build_common<false, double>(h, sa, pa, smax, prm->delta, st, async, P);
}

sai_status sai_psai_build(const sai_split_s* h, const sai_psai_params* prm, cudaStream_t st, bool async,
                          sai_precond_s* P)
{
    if (!h || !prm || !P) return SAI_INVALID_ARG;
    if (prm->lmax < 0 || prm->tol_mode < 0 || prm->tol_mode > 2 || !(prm->delta >= 0.0) || !(prm->tol >= 0.0) ||
        (prm->tol_mode == 2 && prm->lfill < 1) || (prm->growth != 0 && prm->growth != 1))
        return SAI_INVALID_ARG;
    if (prm->precision != SAI_FP64 && prm->precision != SAI_FP32_REFINE64) return SAI_INVALID_ARG;
    SpaiArgs sa = {};
    PsaiArgs pa;
    pa.delta = prm->delta;
    pa.tol = prm->tol;
    pa.tol_mode = prm->tol_mode;
    pa.lmax = prm->lmax;
    pa.lfill = prm->lfill;
    pa.growth = prm->growth;
    if (prm->precision == SAI_FP32_REFINE64)
        return build_common<true, float>(h, sa, pa, Tier2::SCAP, prm->delta, st, async, P);
    return build_common<true, double>(h, sa, pa, Tier2::SCAP, prm->delta, st, async, P);
}

namespace {
__global__ void k_strided(int32_t m, int32_t stride, int32_t* out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)(i * stride);
}

bool config_ok(const sai_build_config& c)
{
    return (c.warps_t0 == 4 || c.warps_t0 == 8) &&
           (c.blocks_per_sm_t12 == 1 || c.blocks_per_sm_t12 == 2 || c.blocks_per_sm_t12 == 4) &&
           (c.heavy_first == 0 || c.heavy_first == 1) && (c.first_tier >= 0 && c.first_tier <= 3);
}
}  // namespace

namespace {
// which: 0 SPAI, 1 PSAI, -1 both
sai_status set_config(const sai_build_config* cfg, int which)
{
    sai_build_config c = cfg ? *cfg : sai_build_config{8, 2, 0, 0, 0.f};
    if (!config_ok(c)) return SAI_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    if (which != 1) g_cfg[0] = c;
    if (which != 0) g_cfg[1] = c;
    return SAI_OK;
}
}  // namespace

sai_status sai_build_set_config_run(const sai_build_config* cfg) { return set_config(cfg, -1); }

sai_status sai_build_autotune_run(const sai_split_s* h, int32_t sai, const sai_spai_params* sp,
                                  const sai_psai_params* pp, cudaStream_t st, sai_build_tuning* out)
{
    if (!h || !out || (sai != 0 && sai != 1) || (sai == 0 && !sp) || (sai == 1 && !pp)) return SAI_INVALID_ARG;
    // parameters are checked by a full-validation build path below (same rules)
    if (sai == 0 && (sp->mn < 1 || sp->mn > MNMAX || sp->max_aug < 0 || sp->key_bits < 1 || sp->key_bits > 31 ||
                     !(sp->delta >= 0.0) || (sp->precision != SAI_FP64 && sp->precision != SAI_FP32_REFINE64)))
        return SAI_INVALID_ARG;
    if (sai == 1 && (pp->lmax < 0 || pp->tol_mode < 0 || pp->tol_mode > 2 || (pp->tol_mode == 2 && pp->lfill < 1) ||
                     (pp->growth != 0 && pp->growth != 1) || !(pp->delta >= 0.0) ||
                     !(pp->tol >= 0.0) || (pp->precision != SAI_FP64 && pp->precision != SAI_FP32_REFINE64)))
        return SAI_INVALID_ARG;
    if (g_num_sms == 0) {
        int dev = 0;
        SAI_CUDA(cudaGetDevice(&dev));
        SAI_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    *out = sai_build_tuning{};
    const int32_t n = h->n;
    if (n <= 0) return SAI_OK;
    int32_t stride = n / 65536 > 1 ? n / 65536 : 1;
    if (n / stride < 4096 && stride > 1) stride = n / 4096 > 1 ? n / 4096 : 1;
    const int32_t m = (n + stride - 1) / stride;
    Buf list;
    SAI_TRY(list.alloc(sizeof(int32_t) * (size_t)m, st, true));
    k_strided<<<SAI_GRID(sai_div_up(m, 256) < 1024u ? sai_div_up(m, 256) : 1024u), 256, 0, st>>>(m, stride,
                                                                                             list.as<int32_t>());
    SAI_CUDA(cudaGetLastError());
    SpaiArgs sa = {};
    PsaiArgs pa = {};
    int32_t smax = Tier2::SCAP;
    double delta = 0.0;
    bool f32 = false;
    if (sai == 0) {
        sa.delta = sp->delta;
        sa.scale = ldexp(1.0, sp->key_bits);
        sa.mn = sp->mn;
        sa.max_aug = sp->max_aug;
        const long long bound = 1 + (long long)sp->mn * sp->max_aug;
        smax = (int32_t)(bound < Tier2::SCAP ? bound : Tier2::SCAP);
        delta = sp->delta;
        f32 = sp->precision == SAI_FP32_REFINE64;
    } else {
        pa.delta = pp->delta;
        pa.tol = pp->tol;
        pa.tol_mode = pp->tol_mode;
        pa.lmax = pp->lmax;
        pa.lfill = pp->lfill;
        pa.growth = pp->growth;
        delta = pp->delta;
        f32 = pp->precision == SAI_FP32_REFINE64;
    }
    cudaEvent_t e0, e1;
    SAI_CUDA(cudaEventCreate(&e0));
    SAI_CUDA(cudaEventCreate(&e1));
    int best = -1;
    // one sampled build (two runs: the first warms the pool and the caches)
    auto run = [&](sai_build_config c, float* ms) -> sai_status {
        for (int rep = 0; rep < 2; ++rep) {
            sai_precond_s P;
            SAI_CUDA(cudaEventRecord(e0, st));
            sai_status r;
            if (sai == 0)
                r = f32 ? build_common<false, float>(h, sa, pa, smax, delta, st, true, &P, list.as<int32_t>(), m, &c)
                        : build_common<false, double>(h, sa, pa, smax, delta, st, true, &P, list.as<int32_t>(), m,
                                                      &c);
            else
                r = f32 ? build_common<true, float>(h, sa, pa, smax, delta, st, true, &P, list.as<int32_t>(), m, &c)
                        : build_common<true, double>(h, sa, pa, smax, delta, st, true, &P, list.as<int32_t>(), m,
                                                     &c);
            if (r != SAI_OK) return r;
            SAI_CUDA(cudaEventRecord(e1, st));
            SAI_CUDA(cudaEventSynchronize(e1));
            SAI_CUDA(cudaEventElapsedTime(ms, e0, e1));
        }
        return SAI_OK;
    };
    auto try_cfg = [&](sai_build_config c) -> sai_status {
        float ms = 0.f;
        const sai_status r = run(c, &ms);
        if (r != SAI_OK) return r;
        c.ms = ms;
        out->cand[out->ncand] = c;
        if (best < 0 || ms < out->cand[best].ms) best = out->ncand;
        ++out->ncand;
        return SAI_OK;
    };
    sai_status r = SAI_OK;
    // the first tier's shape and group size, with the warps per block of
    // the shared-memory tiers (the lane form runs one warp per block)
    for (int ft : {0, 1, 2, 3})
        for (int w : {4, 8})
            if (r == SAI_OK && (ft != 3 || w == 8)) r = try_cfg(sai_build_config{w, 2, 0, ft, 0.f});
    // then the queue order, then the blocks per SM of the global-memory tiers
    if (r == SAI_OK) {
        sai_build_config c = out->cand[best];
        c.heavy_first = 1;
        r = try_cfg(c);
    }
    if (r == SAI_OK) {
        const sai_build_config c0 = out->cand[best];
        for (int b : {1, 4})
            if (r == SAI_OK) {
                sai_build_config c = c0;
                c.blocks_per_sm_t12 = b;
                r = try_cfg(c);
            }
    }
    if (r != SAI_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->chosen = out->cand[best];
    out->sample_columns = m;
    return set_config(&out->chosen, sai);
}

sai_status sai_build_work_reset()
{
    double z[PROF_NSITES * 2] = {};
    SAI_CUDA(cudaMemcpyToSymbol(d_swork, z, sizeof(z)));
    SAI_CUDA(cudaMemcpyToSymbol(d_swork32, z, sizeof(double)));
    return SAI_OK;
}

sai_status sai_build_work_read(double* out, double* flops32)
{
    SAI_CUDA(cudaMemcpyFromSymbol(out, d_swork, sizeof(double) * PROF_NSITES * 2));
    SAI_CUDA(cudaMemcpyFromSymbol(flops32, d_swork32, sizeof(double)));
    return SAI_OK;
}
