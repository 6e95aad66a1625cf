// NTT passes for N = 2^12 (launch entry points declared in ntt_launch.h).
#include "ntt_impl.cuh"
#include "ntt_launch.h"

namespace mmfhe {

void ntt_launch_12(Context &c, const uint64_t *sb, RowMap ms, uint64_t *db, RowMap md, size_t nr, bool inverse,
                   double bytes, const uint64_t *os, const uint64_t *os_sh, cudaStream_t st) {
    ntt_launch_t<12>(c, sb, ms, db, md, nr, inverse, bytes, os, os_sh, st);
}

void modup_launch_12(Context &c, uint64_t *digits, const uint64_t *y, const RowMap &md, const RowGroups &gr,
                     size_t nblk, int nl, int nre, int j0, const uint64_t *m_mont, double bytes_cols,
                     double bytes_rows, double macs, cudaStream_t st) {
    modup_launch_t<12>(c, digits, y, md, gr, nblk, nl, nre, j0, m_mont, bytes_cols, bytes_rows, macs, st);
}

void moddown_launch_12(Context &c, uint64_t *vtmp, const uint64_t *z, const RowMap &mv, const RowGroups &gr,
                       size_t nblk, const CombineArgs &a, int nre, double bytes_cols, double bytes_rows,
                       double macs, const KeyipArgs *ka, cudaStream_t st) {
    moddown_launch_t<12>(c, vtmp, z, mv, gr, nblk, a, nre, bytes_cols, bytes_rows, macs, ka, st);
}

void keyip_p_inv_launch_12(Context &c, uint64_t *z, const KeyipArgs &ka, const RowMap &mz, size_t nr,
                          double bytes_rows, double bytes_cols, const uint64_t *os, const uint64_t *os_sh,
                          cudaStream_t st) {
    keyip_p_inv_launch_t<12>(c, z, ka, mz, nr, bytes_rows, bytes_cols, os, os_sh, st);
}

}  // namespace mmfhe
