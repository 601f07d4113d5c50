"""Physical constants and the data grid used by the oracle (test infrastructure).

The paper fixes f* = c/L and x = 2 pi f / f* (Sec. III, Eq. psd) but not the
numerical values of c, L, the astronomical unit or the year; the values below are the
standard LISA / LDC ones.
"""

C_LIGHT = 299792458.0          # m / s
L_ARM = 2.5e9                  # m, LISA arm length
AU = 1.495978707e11            # m
YEAR = 31557600.0              # s, Julian year
GM_SUN_C3 = 4.925490947e-6     # s, G M_sun / c^3

DT = 15.0                      # s, sampling cadence
N_T = 2 ** 21                  # samples in one observation
TOBS = N_T * DT                # 31,457,280 s
DF = 1.0 / TOBS                # Hz, frequency resolution (Eq. inner's Delta f)

# Instrument-noise levels of the synthetic workloads: amplitudes sqrt(S_oms) in
# m/sqrt(Hz) and sqrt(S_acc) in m s^-2/sqrt(Hz) (Sec. III quotes the LDC2A values
# 7.9e-12 and 2.4e-15; the workloads use 15e-12 and 3e-15).
SQRT_S_OMS = 15e-12
SQRT_S_ACC = 3e-15
