"""Integer constants of the C ABI (the enums and #defines of include/lbm.h).

Plain Python, loading no library: code that only needs the names (the
benchmark's workload tables, its CPU reference arm) imports this module
instead of the ctypes binding.  ``lbm`` re-exports every name.
"""
LBM_OK, LBM_EINVAL, LBM_ESTATE, LBM_ENOMEM, LBM_ECUDA, LBM_ENAN, LBM_ETIMEOUT, LBM_ENOCONV = range(8)
LBM_D2Q9, LBM_D3Q19, LBM_D3Q15, LBM_D3Q27 = 0, 1, 2, 3
LBM_BGK, LBM_MRT, LBM_ELBM, LBM_REG, LBM_SMAG = 0, 1, 2, 3, 4
LBM_F64, LBM_F32, LBM_F32S, LBM_F16S, LBM_BF16S = range(5)
LBM_FIELD_F64, LBM_FIELD_F32 = 0, 1
LBM_ALPHA_NEWTON, LBM_ALPHA_SERIES_GUARDED, LBM_ALPHA_MLP_GUARDED, LBM_ALPHA_FIXED2 = range(4)
LBM_ALPHA_ROOT_GUARDED = 4
LBM_ROUND_DITHER, LBM_ROUND_NEAREST = 0, 1
LBM_PATTERN_AB, LBM_PATTERN_AA = 0, 1
LBM_MASKED_AUTO, LBM_MASKED_NODE, LBM_MASKED_ZRUN = 0, 1, 2
LBM_TRANSFER_STAGED, LBM_TRANSFER_DIRECT = 0, 1
LBM_BC_VELOCITY, LBM_BC_PRESSURE = 1, 2
LBM_BC_EQUILIBRIUM, LBM_BC_ZOUHE, LBM_BC_REGULARIZED = 0, 1, 2
LBM_MLP_FP32, LBM_MLP_BF16_TC = 0, 1
MLP_NPARAM = 1394

NAMES = [k for k in dir() if k.startswith("LBM_")]
