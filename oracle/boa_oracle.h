/*
 * FP64 CPU oracle for the BOA Constrictor hot path.  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the package smoke check and the benchmark's CPU
 * baseline leg may call it.  It shares no code (headers, helpers, tables)
 * with the CUDA library; the two meet only in the weight-file format and in
 * seeded inputs.
 */
#ifndef BOA_ORACLE_H
#define BOA_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_model orc_model;
typedef struct orc_state orc_state;

/* Weight file: 40-byte header then float32 tensors (converted to double). */
int  orc_model_load(const char* path, orc_model** out);   /* 0 on success */
void orc_model_free(orc_model* m);
int  orc_model_dims(const orc_model* m, int* out8);      /* vocab,d,nl,N,K,E,r,ffn_mult */

orc_state* orc_state_new(const orc_model* m);              /* zero conv window and h */
void       orc_state_free(orc_state* s);

/* Step function Phi_theta (paper "Alphabet, sequence, and model"): consume
 * byte s_t, advance the stream cache, write the 256 logits for s_{t+1}. */
void orc_step(const orc_model* m, orc_state* st, int byte, double* logits);

/* Building blocks, exposed so tests can pin each one separately. */
void orc_layernorm(int d, const double* x, const double* g, const double* b, double* y);
void orc_softmax(const double* logits, double* p);                   /* 256 */
void orc_log2_softmax(const double* logits, double* lp);             /* 256 */
void orc_selective_scan(int T, int E, int N, const double* u, const double* delta,
                        const double* A, const double* B, const double* C,
                        const double* D, double* y);                 /* h_0 = 0 */
/* Reverse-mode gradient of sum(dy * y) through orc_selective_scan. */
void orc_selective_scan_grad(int T, int E, int N, const double* u, const double* delta, const double* A,
                             const double* B, const double* C, const double* D, const double* dy, double* du,
                             double* ddelta, double* dA, double* dB, double* dC, double* dD);
void orc_causal_conv(int T, int E, int K, const double* x, const double* w,
                     const double* b, double* out);                  /* zero history, no SiLU */

/* Integer histogram f (sum 2^16, every f >= 1) from probabilities. */
void orc_quantise(const double* p, uint32_t* f);
void orc_quantise_f32(const float* p, uint32_t* f);   /* same rule, float32 arithmetic */
void orc_cdf_from_hist(const uint32_t* f, uint32_t* cdf);           /* 257 entries */

/* Range coder with caller-provided CDFs ([n][257] u32, cdf[0]=0, cdf[256]=2^16). */
size_t orc_coded_bound(size_t n_symbols);
int orc_encode_cdfs(size_t n, const uint32_t* cdfs, const uint8_t* syms, uint8_t* out,
                    size_t cap, size_t* size, uint64_t* straddles);
int orc_decode_cdfs(size_t n, const uint32_t* cdfs, const uint8_t* in, size_t size,
                    uint8_t* syms);

/* Whole method on one stream: out = [raw first byte][coded bytes incl. 4-byte flush]. */
size_t orc_max_compressed_size(size_t len);
int orc_compress_stream(const orc_model* m, const uint8_t* in, size_t len, uint8_t* out,
                        size_t cap, size_t* size);
int orc_decompress_stream(const orc_model* m, const uint8_t* in, size_t size, size_t len,
                          uint8_t* out);
/* Teacher-forced per-step outputs for steps t = 0..len-2 (predicting byte t+1). */
int orc_logprobs(const orc_model* m, const uint8_t* in, size_t len, double* log2p);  /* [(len-1)][256] */
int orc_cdfs(const orc_model* m, const uint8_t* in, size_t len, uint32_t* cdfs);     /* [(len-1)][257] */

/* Many streams, one OpenMP thread per stream (the paper's CPU path). */
int orc_compress_batch(const orc_model* m, size_t n, const uint8_t* const* ins, const size_t* lens,
                       uint8_t* const* outs, const size_t* caps, size_t* sizes, int n_threads);

int orc_decompress_batch(const orc_model* m, size_t n, const uint8_t* const* ins, const size_t* sizes,
                         const size_t* lens, uint8_t* const* outs, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
