/*
 * polar_oracle.h -- TEST INFRASTRUCTURE ONLY (see polar_oracle.c).
 * Declarations of the plain CPU oracle.  Shares nothing with the CUDA library.
 */
#ifndef POLAR_ORACLE_H
#define POLAR_ORACLE_H
#include <stdint.h>

/* a polar code: N = 2^n, K = |A| (includes the c CRC bits), frozen[i] = 1 for
 * i not in A, punct[i] = 1 for a position that is not transmitted (or NULL) */
typedef struct {
    int N;
    int K;
    int crc_len;
    uint32_t crc_poly;
    int systematic;
    const uint8_t *frozen;
    const uint8_t *punct;
} orc_code;

enum { ORC_PRUNE_R0 = 1, ORC_PRUNE_R1 = 2, ORC_PRUNE_REP = 4, ORC_PRUNE_SPC = 8 };

/* tree pruning: enabled node types, size limits (0 = none; spc_max = 4 is
 * SPC4, rep_max = 8 is REP8-), flip depths (0 = every position), and the
 * smallest node of more than one leaf that is pruned (0, 1 or 2 = any;
 * smaller nodes are decoded leaf by leaf)                                  */
typedef struct {
    uint32_t mask;
    int rep_max;
    int spc_max;
    int r1_t;
    int spc_t;
    int r1_max;
    int node_min;
} orc_pruning;

enum { ORC_NODE_INTERNAL = 0, ORC_NODE_R0 = 1, ORC_NODE_R1 = 2, ORC_NODE_REP = 3, ORC_NODE_SPC = 4 };
enum { ORC_F32 = 0, ORC_I16 = 1, ORC_I8 = 2, ORC_IWIDE = 3, ORC_EXACT = 4 };
enum { ORC_MODE_F32 = 0, ORC_MODE_FIXED = 1, ORC_MODE_EXACT = 2 };
enum { ORC_ALGO_SC = 0, ORC_ALGO_CASCL = 1, ORC_ALGO_PA = 2, ORC_ALGO_FA = 3 };

/* work counters: f/g element operations summed over active paths, node steps
 * (leaves and pruned nodes), steps that had to discard candidates, the total
 * number of candidates offered, and decode stages run                      */
typedef struct {
    long long fg_elems;
    long long node_steps;
    long long sorts;
    long long cand_total;
    long long stages;
} orc_stats;

void orc_polar_transform(int N, uint8_t *v);
uint32_t orc_crc(const uint8_t *bits, int nbits, int c, uint32_t poly);
int orc_encode(const orc_code *cd, const uint8_t *info, uint8_t *x);
void orc_encode_batch(const orc_code *cd, int n_frames, const uint8_t *info, uint8_t *x, int *rc);
void orc_ga_reliability(int N, const uint8_t *punct, double sigma2, double *z_leaves);
void orc_ga_frozen(int N, int K, int K_info, const uint8_t *punct, double design_ebn0_db,
                   uint8_t *frozen, double *z_out);
void orc_qup_pattern(int N, int P, uint8_t *punct);
void orc_de_bms(int N, const uint8_t *punct, int m, const double *q, const double *p, int mu, double *pe);
int orc_de_awgn_channel(double sigma2, int mu, double *q, double *p);
void orc_de_reliability(int N, const uint8_t *punct, double sigma2, int mu, double *pe);
void orc_de_frozen(int N, int K, int K_info, const uint8_t *punct, double design_ebn0_db, int mu,
                   uint8_t *frozen, double *pe_out);
int orc_decode(const orc_code *cd, const double *llr, int L, int algo, const orc_pruning *pr,
               int mode, int wide_frac, double wide_q, uint8_t *info_out, int32_t *status,
               double *pm_out, uint8_t *paths_out, orc_stats *st);
int orc_decode_batch(const orc_code *cd, const double *llr, int n_frames, int L, int algo,
                     const orc_pruning *pr, int mode, int wide_frac, double wide_q, uint8_t *info_out,
                     int32_t *status, double *pm_out, orc_stats *st);
int orc_sc_plain(const orc_code *cd, const double *llr, const orc_pruning *pr, int mode, int wide_frac,
                 double wide_q, uint8_t *x_out);
int orc_node_list(const orc_code *cd, const orc_pruning *pr, int32_t *out);

#endif
