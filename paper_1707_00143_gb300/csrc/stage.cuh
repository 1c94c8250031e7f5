// stage.cuh -- staged gathers of wide base rows for the search (Alg. 1).
//
// The rows an expansion measures are copied from global into a per-warp ring
// of shared-memory slots by the bulk-copy (TMA) engine, one untiled
// cp.async.bulk per row, each completing on the slot's mbarrier.  One lane
// issues the first `nb` rows of the list at once, so they are all in flight
// together; the warp then measures row c from its slot (the same lane slices
// and sums as the register gather, so the same keys) and refills the slot
// with row c + nb.  Rows past the ring are prefetched into L2 first, so the
// refills come from L2.  The keys are the register gather's, so the search's
// steps and results are too.  Rows with a tensor map over them (the BF16 /
// FP8 / U8 copies of rows of at most 2 KB) are gathered four per copy
// instead: a slot holds the four rows of one tile::gather4.
//
// Measured (GIST-shaped 1M x 960, k = 100, L = 300, one query alone): a
// staged row costs ~0.4 us whether it is 960 or 3,840 bytes and whatever the
// ring size (2..16) or the issuing lanes -- bulk copies of rows picked at
// random complete about one after another -- so an 8-bit expansion (46 rows)
// takes 17.8 us staged against 7.1 us in registers (8 rows in flight per
// lane group), while FP32 rows, two in flight per group in registers, take
// the same 20.4 us either way; in a batch the staged FP32 form with 4 slots
// frees the registers the gather held and runs 7-38 % faster.  Four-row
// gathers take the 8-bit expansion to 13.4 us: the rows of one gather also
// arrive one after another.  The launch therefore stages only FP32-sized
// rows (more than 2 KB) by default.
//
// Every wait is bounded (STAGE_TIMEOUT_NS).  A copy that never lands marks
// the warp failed: it drains (again bounded) the copies it still has in
// flight, stops issuing, measures nothing more (keys +inf), raises bit 1 of
// the launch's error flag and the query reports NSG_ECUDA.
#pragma once

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nsg {

constexpr uint64_t STAGE_TIMEOUT_NS = 4000000000ull;  // far beyond any legitimate copy
constexpr int STAGE_MAX_SLOTS = 32;

// Per-warp staging region: nb mbarriers, two state words (slot parity bits,
// failure), then (128-byte aligned) the ring of nb slots of `slot_bytes`.
struct StageRef {
    unsigned char *ring;
    uint64_t *bar;
    uint32_t *state;  // [0] parity of each slot's next phase, [1] failed
    int nb;           // mbarriers = slots
    int ring_bytes;
    int *err;         // launch flag (bit 1: a staged copy never landed), nullable
};

__host__ __device__ inline int stage_ring_offset(int nb) { return (nb * 8 + 8 + 15) & ~15; }
// the region of nb slots of slot_bytes, with room to align the ring to 128 bytes
__host__ __device__ inline size_t stage_bytes(int nb, int slot_bytes) {
    return (size_t)stage_ring_offset(nb) + 112 + (size_t)nb * slot_bytes;
}
// a slot of four rows for the gathered copies (tensor copies land on 128-byte boundaries)
__host__ __device__ inline int stage_group_bytes(int row_bytes) { return (4 * row_bytes + 127) & ~127; }

// Carve and initialise the warp's region (once per kernel, before any use).
__device__ inline StageRef stage_init(unsigned char *p, int nb, int slot_bytes, int *err) {
    StageRef r;
    r.bar = reinterpret_cast<uint64_t *>(p);
    r.state = reinterpret_cast<uint32_t *>(r.bar + nb);
    const uintptr_t ring = reinterpret_cast<uintptr_t>(p + stage_ring_offset(nb));
    r.ring = reinterpret_cast<unsigned char *>((ring + 127) & ~uintptr_t(127));
    r.nb = nb;
    r.ring_bytes = nb * slot_bytes;
    r.err = err;
    if (lane_id() == 0) {
        for (int i = 0; i < nb; ++i) tc::mbar_init(r.bar + i, 1);
        r.state[0] = 0;
        r.state[1] = 0;
        tc::fence_barrier_init();
    }
    __syncwarp();
    return r;
}

// Bounded wait for the phase of the given parity of one slot's barrier.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = tc::globaltimer();
    for (uint32_t spin = 1;; ++spin) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0 && tc::globaltimer() - t0 > limit_ns) return false;
    }
}

// Distance functor over staged rows: D is a register-gather functor with one
// row per warp (G = 32) providing row_addr, row_bytes and row_smem.  With a
// tensor map over D's rows (map != nullptr) a slot holds four rows fetched by
// one tile::gather4 copy (the last group repeats its last row); otherwise a
// slot holds one row fetched by one bulk copy.
template <class D>
struct DistStaged {
    D reg;
    StageRef sr;
    int nb, rb;               // slots, bytes per row
    const CUtensorMap *map;   // rows four per copy through this map, or nullptr

    __device__ __forceinline__ int slot_bytes() const { return map ? stage_group_bytes(rb) : rb; }

    // the copy of group gi (rows gi * R .. of ids[0..m)) into `slot`; lane 0
    __device__ __forceinline__ void issue(int slot, const int *ids, int gi, int m) const {
        unsigned char *dst = sr.ring + (size_t)slot * slot_bytes();
        if (map) {
            const int j = gi * 4, last = m - 1;
            const int y0 = ids[j], y1 = ids[j + 1 < m ? j + 1 : last], y2 = ids[j + 2 < m ? j + 2 : last],
                      y3 = ids[j + 3 < m ? j + 3 : last];
            tc::mbar_expect_tx(sr.bar + slot, (uint32_t)(4 * rb));
            tc::tma_gather4(dst, map, sr.bar + slot, 0, y0, y1, y2, y3);
        } else {
            tc::mbar_expect_tx(sr.bar + slot, (uint32_t)rb);
            tc::bulk_load(dst, reg.row_addr(ids[gi]), (uint32_t)rb, sr.bar + slot);
        }
    }

    __device__ void operator()(const int *ids, int m, uint64_t *keys) const {
        const unsigned lane = lane_id();
        const int R = map ? 4 : 1;
        const int ng = (m + R - 1) / R;
        uint32_t bits = sr.state[0];
        const bool failed = sr.state[1] != 0;
        __syncwarp();
        int gi = 0;
        if (!failed) {
            const int first = ng < nb ? ng : nb;
            if (lane == 0)
                for (int j = 0; j < first; ++j) issue(j, ids, j, m);
            if (ng > nb) prefetch_rows_l2(reg.row_addr(0), rb, ids + nb * R, m - nb * R);
            // no lane waits on a copy before lane 0 has issued it: a diverged
            // warp may run the waiting lanes' spin ahead of the issuing lane
            __syncwarp();
            int slot = 0;
            for (; gi < ng; ++gi) {
                const bool ok = __all_sync(NSG_FULL, stage_wait(sr.bar + slot, (bits >> slot) & 1u, STAGE_TIMEOUT_NS));
                if (!ok) break;
                bits ^= 1u << slot;
                const unsigned char *src = sr.ring + (size_t)slot * slot_bytes();
                for (int r = 0; r < R; ++r) {
                    const int c = gi * R + r;
                    if (c >= m) break;
                    const float d2 = reg.row_smem(src + (size_t)r * rb);
                    if (lane == 0) keys[c] = make_key(d2, ids[c]);
                }
                __syncwarp();  // every lane has read the slot
                if (lane == 0 && gi + nb < ng) {
                    tc::fence_proxy_async_smem();
                    issue(slot, ids, gi + nb, m);
                }
                __syncwarp();
                slot = slot + 1 == nb ? 0 : slot + 1;
            }
            if (gi < ng) {  // a copy never landed: drain the ones in flight (bounded), then stop
                const int issued = ng < gi + nb ? ng : gi + nb;
                for (int j = gi; j < issued; ++j) {
                    const int sl = j % nb;
                    stage_wait(sr.bar + sl, (bits >> sl) & 1u, STAGE_TIMEOUT_NS / 4);
                    bits ^= 1u << sl;
                }
                if (lane == 0) {
                    sr.state[1] = 1;
                    if (sr.err) atomicOr(sr.err, 2);
                }
            }
        }
        for (int j = gi * R + (int)lane; j < m; j += 32) keys[j] = make_key(__int_as_float(0x7f800000), ids[j]);
        __syncwarp();
        if (lane == 0) sr.state[0] = bits;
        __syncwarp();
    }
    // operator() prefetches the rows past its ring itself
    __device__ __forceinline__ void prefetch(const int *, int) const {}
    __device__ __forceinline__ void prefetch_all(const int *ids, int m) const { reg.prefetch_all(ids, m); }
};

// Slots of reg's rows (one row each, or groups of four with a map) that ring
// `sr` holds, at most its barriers (0: not one fits).
template <class D>
__device__ __forceinline__ int stage_slots(const D &reg, const StageRef &sr, bool grouped = false) {
    const int nb = sr.ring_bytes / (grouped ? stage_group_bytes(reg.row_bytes()) : reg.row_bytes());
    return nb < sr.nb ? nb : sr.nb;
}

}  // namespace nsg
