// Per-ring-dimension launch entry points of the NTT passes (defined in
// ntt_l10.cu .. ntt_l16.cu, one translation unit per log N).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"

namespace mmfhe {

#define MMFHE_NTT_ENTRY_DECL(L)                                                                                   \
    void ntt_launch_##L(Context &c, const uint64_t *sb, RowMap ms, uint64_t *db, RowMap md, size_t nr,          \
                        bool inverse, double bytes, const uint64_t *os, const uint64_t *os_sh, cudaStream_t st); \
    void modup_launch_##L(Context &c, uint64_t *digits, const uint64_t *y, const RowMap &md, const RowGroups &gr, \
                          size_t nblk, int nl, int nre, int j0, const uint64_t *m_mont, double bytes_cols,     \
                          double bytes_rows, double macs, cudaStream_t st);                                     \
    void moddown_launch_##L(Context &c, uint64_t *vtmp, const uint64_t *z, const RowMap &mv, const RowGroups &gr, \
                            size_t nblk, const CombineArgs &a, int nre, double bytes_cols, double bytes_rows,  \
                            double macs, const KeyipArgs *ka, cudaStream_t st);                                 \
    void keyip_p_inv_launch_##L(Context &c, uint64_t *z, const KeyipArgs &ka, const RowMap &mz, size_t nr,      \
                                double bytes_rows, double bytes_cols, const uint64_t *os, const uint64_t *os_sh, \
                                cudaStream_t st);
MMFHE_NTT_ENTRY_DECL(10)
MMFHE_NTT_ENTRY_DECL(11)
MMFHE_NTT_ENTRY_DECL(12)
MMFHE_NTT_ENTRY_DECL(13)
MMFHE_NTT_ENTRY_DECL(14)
MMFHE_NTT_ENTRY_DECL(15)
MMFHE_NTT_ENTRY_DECL(16)
#undef MMFHE_NTT_ENTRY_DECL

}  // namespace mmfhe
