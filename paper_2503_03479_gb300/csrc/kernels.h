// kernels.h -- launchers of the libasift kernels (internal).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "asift.h"

namespace asift {

struct DevView;
struct DevLevel;
struct Candidate;
struct SlotKp;

// warp.cu
void warp_strip_widths(const asift_view_desc &v, int tw, int *cw, int *bw);
int warp_tile_width(const asift_view_desc &v);
void warp_lane_layout(long long cq, long long sq, int *lanes_x, int *pitch);
cudaError_t launch_u8_to_f32(const uint8_t *src, int pitch, int W, int H, float *dst, int dpitch, cudaStream_t s);
struct ImageConv;
cudaError_t launch_convert_images(const ImageConv *d_list, int n, long long max_px, cudaStream_t s);
int tilt_filter_pitch(int K);
cudaError_t launch_tilt_filter(const DevView *d_views, int n_views, int max_wv, cudaStream_t s);
struct DevRotGroup;
int warp_seg_width_default();
bool warp_seg_width_ok(int seg_w, int hk_max);
void build_rot_groups(const asift_view_desc *h, const DevView *dv, int nv, bool per_view, int seg_w,
                      std::vector<DevRotGroup> &out, int *n_tiles, int *hk_max);
cudaError_t launch_warp(const DevRotGroup *d_groups, int n_groups, const DevView *d_views, int n_tiles, int seg_w,
                        int hk_max, uint8_t *u8, uint8_t *mask, float *f32, cudaStream_t s, int grid = 0);
int warp_nn_strip_width(const asift_view_desc &v, int tw);
// warp_precise.cu
int warp_lz_strip_width(const asift_view_desc &v, int tw, int a);
cudaError_t launch_warp_lanczos(int a, const DevView *d_views, int n_views, int n_tiles, int cw_max, uint8_t *u8,
                                uint8_t *mask, float *f32, cudaStream_t s);
cudaError_t launch_warp_nn(const DevView *d_views, int n_views, int n_tiles, int cw_max, uint8_t *u8, uint8_t *mask,
                           float *f32, cudaStream_t s, int grid = 0);

// orb.cu
struct DetItem;
cudaError_t launch_mask_rows(const DevLevel *d_lv, int nv, int n_levels, int rows0, int max_h1, int32_t *row_lo,
                             int32_t *row_hi, int32_t *unit, cudaStream_t s);
cudaError_t launch_pyramid(const DevLevel *d_lv, int n, int n_tiles, const int32_t *unit, cudaStream_t s, int grid = 0);
cudaError_t launch_detect(const DevLevel *d_lv, int n, int n_tiles, int thr, Candidate *cand, int32_t *count,
                          const int32_t *row_lo, const int32_t *row_hi, const int32_t *unit, DetItem *list,
                          int32_t *list_count, cudaStream_t s, int grid = 0);
size_t select_smem_bytes();
cudaError_t launch_select(const DevLevel *d_lv, int n, const Candidate *cand, const int32_t *count, int n_features,
                          SlotKp *slots, int32_t *taken, int32_t *status, cudaStream_t s);
cudaError_t launch_pool_scan(const int32_t *taken, int n_views, int n_levels, const int32_t *group_first_view,
                             int n_groups, int n_features, int32_t *pool_off, int32_t *view_count,
                             int32_t *view_off, int32_t *group_total, cudaStream_t s);
cudaError_t launch_orient_brief(const DevLevel *d_lv, int n_views, int n_levels, int n_features, int v_begin,
                                int v_end, const SlotKp *slots, const int32_t *taken, const int32_t *pool_off,
                                const int *pattern, const long long *bins, asift_keypoint *kp, uint4 *desc,
                                cudaStream_t s);

// match.cu
struct MatchProblem;
struct MatchTuning;
int hamming_splits_alloc(int nt_cap);
size_t hamming_partial_bytes(int nq, int nt);
int pair_blocks(int nq);
int match_max_problems();
void match_problem_init(MatchProblem &P, const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                        const int32_t *d_nt, void *region, int s_alloc, asift_match *out, uint8_t *accept,
                        int32_t *n_acc);
void match_problems_offsets(MatchProblem *probs, int n, int *total_q, int *total_blk);
cudaError_t launch_match(const MatchProblem *d_probs, int n_probs, const MatchProblem &single, int total_q,
                         bool any_train, int num, int den, const MatchTuning &tune, cudaStream_t s);
cudaError_t launch_merge(const MatchProblem *d_probs, int n_probs, const MatchProblem &single, int total_q, int num,
                         int den, cudaStream_t s);
cudaError_t launch_hamming(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                           const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                           int32_t *n_acc, void *part, cudaStream_t s);
cudaError_t launch_hamming_noalloc(const uint8_t *q, int nq, const int32_t *d_nq, const uint8_t *t, int nt,
                                   const int32_t *d_nt, int num, int den, asift_match *out, uint8_t *accept,
                                   int32_t *n_acc, cudaStream_t s);
cudaError_t launch_pairs(const MatchProblem *d_probs, int n_probs, const MatchProblem &single, int total_blk,
                         int32_t *block_count, const DevLevel *lv, int nv, int32_t *status, cudaStream_t s);
// eval.cu
size_t eval_workspace_bytes(int cap, int n_hyp);
cudaError_t launch_eval(const asift_pair_match *d_pairs, const int32_t *d_n, int cap, const double *h_H_true,
                        double th_sq, const uint32_t *d_rnd, int n_hyp, double ransac_th_sq,
                        asift_pair_match *d_unique, uint8_t *d_inlier, int32_t *d_hyp_counts,
                        asift_eval_result *d_res, void *d_ws, cudaStream_t s);
// sift.cu
size_t sift_workspace_bytes(int W, int H, int max_kp);
cudaError_t launch_sift(const uint8_t *d_img, int W, int H, int pitch, int max_kp, asift_sift_kp *d_kp, float *d_desc,
                        int32_t *d_n, void *d_ws, cudaStream_t s);
// sift_match.cu
size_t sift_match_workspace_bytes(int nq, int nt);
cudaError_t launch_sift_match(const float *q, int nq, const int32_t *d_nq, const float *t, int nt, const int32_t *d_nt,
                              double ratio, const asift_sift_kp *kq, const asift_sift_kp *kt, asift_l2_match *out,
                              asift_pair_match *pairs, int cap, int32_t *d_n, void *ws, cudaStream_t s);
size_t scale_coeff_workspace_bytes(int cap);
cudaError_t launch_scale_coeff(const asift_pair_match *d_pairs, const int32_t *d_n, int cap, double *d_f, void *d_ws,
                               cudaStream_t s);
size_t eval_batch_workspace_bytes(const int *caps, int n, int n_hyp);
cudaError_t launch_eval_batch(asift_pair_match *const *pairs, int32_t *d_ns, const int *caps, int n,
                              const double *h_H_true, double th_sq, const uint32_t *d_rnd, int n_hyp,
                              double ransac_th_sq, void *d_ws, cudaStream_t s);
void eval_batch_outputs(void *d_ws, const int *caps, int n, int n_hyp, int i, asift_pair_match **unique,
                        uint8_t **inlier, int32_t **counts, asift_eval_result **res);
int view_count_max_views();
cudaError_t launch_view_counts(const asift_keypoint *kp, const uint8_t *accept, const int32_t *d_nq, int nq_cap,
                               int view0, int n_views, int32_t *counts, int32_t *best, cudaStream_t s);

// match_tc.cu (tensor-core matcher; same partials and merge as match.cu)
bool tc_match_available();
size_t tc_expanded_bytes(long long rows);
cudaError_t launch_expand(const uint8_t *packed, uint8_t *out, const int32_t *d_first, int n_per_view,
                          const int32_t *d_count, long long cap_rows, int n_groups, cudaStream_t s);
cudaError_t launch_match_tc(const uint8_t *qbase, const uint8_t *qexp, long long q_rows, const uint8_t *tbase,
                            const uint8_t *texp, long long t_rows, const MatchProblem *d_probs, int n_probs,
                            const MatchProblem &single, int total_q, int num, int den, const MatchTuning &tune,
                            int32_t *status, cudaStream_t s);

// dwarp.cu
struct DiffView;
int dwarp_tile_width(bool backward);
void dwarp_strip_widths(int tw, double t_max, int K, int *cw, int *bw);
int dwarp_tiles(int Wv, int Hv, int tw, int *ntx);
struct DiffPrep;
cudaError_t launch_dwarp(bool backward, const DiffView *d_views, DiffPrep *d_prep, int n_views, int n_tiles,
                         int cw_max, int bw_max, int32_t *status, cudaStream_t s);
struct WarpSeg {            // one view of a flat view buffer
    long long off, count;
};
struct AdamArgs {           // one Adam step of the view parameters (t, phi, tx, ty)
    double lr[4];
    double scale;           // decay^step
    double c1, c2;          // bias corrections 1 - b1^(step+1), 1 - b2^(step+1)
    double t_lo, t_hi;
};
cudaError_t launch_warp_loss(const WarpSeg *d_segs, int n, long long max_count, const float *v, const float *target,
                             double *loss, float *vbar, cudaStream_t s);
cudaError_t launch_warp_adam(int n, double *params, const double *grad, double *m, double *v, const AdamArgs &a,
                             cudaStream_t s);

// tables.cpp (host; each table generated from its written definition)
void make_view_desc(int H, int W, double t, double phi_deg, int k, int j, double scale, asift_view_desc *v);
int view_table(int H, int W, int kmax, asift_view_desc *out, int cap);
int view_table_scaled(int H, int W, int kmax, double ds, asift_view_desc *out, int cap);
int level_size(int n0, int l);
void make_pattern(uint64_t seed, int8_t pat[30][256][4]);
void make_bin_table(long long e[30][2]);

}  // namespace asift
