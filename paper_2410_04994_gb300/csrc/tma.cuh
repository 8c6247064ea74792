// Tensor-memory-accelerator (TMA) copies and mbarrier waits in inline PTX.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace shg {

SHG_D unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

SHG_D void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// Make the barrier's initialisation visible to the asynchronous (TMA) proxy.
SHG_D void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

SHG_D void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

SHG_D bool mbar_try_wait(uint64_t* bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `phase`: false if the barrier did not complete within
// `max_iter` polls (each poll may itself suspend for a short while).
SHG_D bool mbar_wait_bounded(uint64_t* bar, unsigned phase, unsigned max_iter) {
    for (unsigned it = 0; it < max_iter; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// 3-D tiled tensor copy global -> shared, completing on `bar`.  The box's
// innermost coordinate must keep the copy 16-byte aligned.
SHG_D void tma_load_3d(void* dst, const CUtensorMap* tmap, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace shg
