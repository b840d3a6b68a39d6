// Instantiates the re-rank kernels for one (row kind, R) pair, chosen by
// -DTACO_INST_BF16=<0 FP32 | 1 BF16 | 2 FP8> -DTACO_INST_R=<1|4|16>; the build compiles this
// file nine times. The cluster kernel takes both (FP32 and BF16 rows); the select pass takes
// the row kind only and is instantiated in the R = 1 units. FP8 rows have the select pass only.
#include "taco_rerank.cuh"
#include "taco_select.cuh"

#ifndef TACO_INST_BF16
#define TACO_INST_BF16 0
#endif
#ifndef TACO_INST_R
#define TACO_INST_R 1
#endif

#define TACO_CAT_(a, b, c, d) a##b##c##d
#define TACO_CAT(a, b, c, d) TACO_CAT_(a, b, c, d)
#define TACO_FN TACO_CAT(launch_rerank_b, TACO_INST_BF16, _r, TACO_INST_R)
#define TACO_CAT2_(a, b) a##b
#define TACO_CAT2(a, b) TACO_CAT2_(a, b)
#define TACO_FN2 TACO_CAT2(launch_select_b, TACO_INST_BF16)

namespace taco {

#if TACO_INST_BF16 != 2
cudaError_t TACO_FN(int G, const RerankParams& P, int cluster, int64_t nq, size_t smem,
                    cudaStream_t st) {
    constexpr bool kBf16 = TACO_INST_BF16 != 0;
    switch (G) {
        case 4: return launch_rerank_t<4, TACO_INST_R, kBf16>(P, cluster, nq, smem, st);
        case 8: return launch_rerank_t<8, TACO_INST_R, kBf16>(P, cluster, nq, smem, st);
        case 16: return launch_rerank_t<16, TACO_INST_R, kBf16>(P, cluster, nq, smem, st);
        case 32: return launch_rerank_t<32, TACO_INST_R, kBf16>(P, cluster, nq, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

#endif

#if TACO_INST_R == 1   // the select pass has no register lists: one unit per row kind
cudaError_t TACO_FN2(int G, const RerankParams& P, int64_t nq, size_t smem, cudaStream_t st) {
    constexpr int kRow = TACO_INST_BF16;
    switch (G) {
        case 4: return launch_select_rerank_t<4, kRow>(P, nq, smem, st);
        case 8: return launch_select_rerank_t<8, kRow>(P, nq, smem, st);
        case 16: return launch_select_rerank_t<16, kRow>(P, nq, smem, st);
        case 32: return launch_select_rerank_t<32, kRow>(P, nq, smem, st);
        default: return cudaErrorInvalidValue;
    }
}
#endif

}  // namespace taco
