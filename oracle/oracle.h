/*
 * Oracle declarations (test infrastructure only; see oracle.c).  This header
 * belongs to the oracle alone: the CUDA library neither includes nor shares it.
 */
#ifndef BINARIZE_ORACLE_H
#define BINARIZE_ORACLE_H
#include <stdint.h>

#define ORACLE_SAUVOLA 0
#define ORACLE_NIBLACK 1
/* 2 is the quantile method */
#define ORACLE_WOLF 3
#define ORACLE_FENG 4
#define ORACLE_RAIS 5
#define ORACLE_NICK 6
#define ORACLE_PHANSALKAR 7

void oracle_window_params(int32_t h, int32_t w, int32_t *l, int32_t *r,
                          int32_t *o, int32_t *u);
int oracle_window_sums_bruteforce(const uint8_t *img, int64_t H, int64_t W,
                                  int64_t pitch, int32_t h, int32_t w,
                                  uint32_t *S1, uint64_t *S2, uint32_t *n);
int oracle_window_sums_integral(const uint8_t *img, int64_t H, int64_t W,
                                int64_t pitch, int32_t h, int32_t w,
                                uint32_t *S1, uint64_t *S2, uint32_t *n);
int oracle_window_sums_recursive(const uint8_t *img, int64_t H, int64_t W,
                                 int64_t pitch, int32_t h, int32_t w,
                                 uint32_t *S1, uint64_t *S2, uint32_t *n);
double oracle_threshold(int32_t method, uint32_t S1, uint64_t S2, uint32_t n,
                        double k, double R);
float oracle_threshold_f32(int32_t method, uint32_t S1, uint64_t S2, uint32_t n,
                           float k, float R);
uint8_t oracle_sauvola_bit_paper_order(uint32_t I, uint32_t S1, uint64_t S2,
                                       uint32_t n, double k, double R);
uint8_t oracle_sauvola_bit_exact(uint32_t I, uint32_t S1, uint64_t S2,
                                 uint32_t n, int64_t kn, int64_t kd,
                                 int64_t Rn, int64_t Rd);
void oracle_pack_bits(const uint8_t *bits, int64_t H, int64_t W, uint8_t *out,
                      int64_t out_pitch);
int oracle_binarize(int32_t method, const uint8_t *img, int64_t H, int64_t W,
                    int64_t pitch, int32_t h, int32_t w, double k, double R,
                    uint8_t *bits, uint8_t *out, int64_t out_pitch);
int oracle_binarize_parallel(int32_t method, const uint8_t *img, int64_t H,
                             int64_t W, int64_t pitch, int32_t h, int32_t w,
                             double k, double R, uint8_t *out, int64_t out_pitch,
                             int32_t nthreads);
int32_t oracle_openmp_max_threads(void);
int oracle_window_quantile_sort(const uint8_t *img, int64_t H, int64_t W,
                                int64_t pitch, int32_t h, int32_t w,
                                int32_t q_num, int32_t q_den, uint8_t *Q);
int oracle_window_quantile_count(const uint8_t *img, int64_t H, int64_t W,
                                 int64_t pitch, int32_t h, int32_t w,
                                 int32_t q_num, int32_t q_den, uint8_t *Q);
int oracle_window_quantile_sliding(const uint8_t *img, int64_t H, int64_t W,
                                   int64_t pitch, int32_t h, int32_t w,
                                   int32_t q_num, int32_t q_den, uint8_t *Q,
                                   int32_t nthreads);
int oracle_binarize_quantile(const uint8_t *img, int64_t H, int64_t W,
                             int64_t pitch, int32_t h, int32_t w, int32_t q_num,
                             int32_t q_den, int32_t offset, uint8_t *bits,
                             uint8_t *out, int64_t out_pitch, int32_t nthreads);
void oracle_threshold_array(int32_t method, const uint32_t *S1, const uint64_t *S2,
                            const uint32_t *n, int64_t count, double k, double R,
                            double *t);
void oracle_threshold_f32_array(int32_t method, const uint32_t *S1, const uint64_t *S2,
                                const uint32_t *n, int64_t count, float k, float R,
                                float *t);
void oracle_sauvola_bits_exact_array(const uint8_t *img, const uint32_t *S1,
                                     const uint64_t *S2, const uint32_t *n,
                                     int64_t count, int64_t kn, int64_t kd,
                                     int64_t Rn, int64_t Rd, uint8_t *bits);
void oracle_sauvola_bits_paper_order_array(const uint8_t *img, const uint32_t *S1,
                                           const uint64_t *S2, const uint32_t *n,
                                           int64_t count, double k, double R,
                                           uint8_t *bits);
void oracle_window_sums_at(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                           int32_t h, int32_t w, const int64_t *ii,
                           const int64_t *jj, int64_t count, uint32_t *S1,
                           uint64_t *S2, uint32_t *n);
void oracle_window_quantile_at(const uint8_t *img, int64_t H, int64_t W,
                               int64_t pitch, int32_t h, int32_t w, int32_t q_num,
                               int32_t q_den, const int64_t *ii, const int64_t *jj,
                               int64_t count, uint8_t *Q);
int oracle_global_stats(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                        double *stats, uint64_t *sums);
double oracle_threshold_ext(int32_t method, uint32_t S1, uint64_t S2, uint32_t n,
                            const double *prm, const double *glob);
void oracle_threshold_ext_array(int32_t method, const uint32_t *S1, const uint64_t *S2,
                                const uint32_t *n, int64_t count, const double *prm,
                                const double *glob, double *t);
int oracle_binarize_ext(int32_t method, const uint8_t *img, int64_t H, int64_t W,
                        int64_t pitch, int32_t h, int32_t w, const double *prm,
                        uint8_t *bits, uint8_t *out, int64_t out_pitch);
int oracle_window_minmax_bruteforce(const uint8_t *img, int64_t H, int64_t W,
                                    int64_t pitch, int32_t h, int32_t w,
                                    uint8_t *mn, uint8_t *mx);
int oracle_window_minmax_deque(const uint8_t *img, int64_t H, int64_t W,
                               int64_t pitch, int32_t h, int32_t w,
                               uint8_t *mn, uint8_t *mx);
int oracle_binarize_bernsen(const uint8_t *img, int64_t H, int64_t W,
                            int64_t pitch, int32_t h, int32_t w,
                            int32_t contrast_limit, uint8_t *bits,
                            uint8_t *out, int64_t out_pitch);
void oracle_window_minmax_at(const uint8_t *img, int64_t H, int64_t W,
                             int64_t pitch, int32_t h, int32_t w,
                             const int64_t *ii, const int64_t *jj, int64_t count,
                             uint8_t *mn, uint8_t *mx);
int oracle_haar_bruteforce(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                           const int32_t *row_len, const int32_t *row_wt, int32_t n_row,
                           const int32_t *col_len, const int32_t *col_wt, int32_t n_col,
                           int32_t *out);
int oracle_haar_integral(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                         const int32_t *row_len, const int32_t *row_wt, int32_t n_row,
                         const int32_t *col_len, const int32_t *col_wt, int32_t n_col,
                         int32_t *out);
#endif
