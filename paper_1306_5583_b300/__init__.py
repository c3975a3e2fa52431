"""B300-native (sm_103a) data-parallel hot path of the generic SMC iteration
of vSMC (Zhou, arXiv 1306.5583): per-particle move, log-weight update,
log-sum-exp normaliser with the ESS test, resampling and the evidence
estimators, behind the C ABI declared in include/smc.h.

``paper_1306_5583_b300.smc`` is the thin Python binding over that ABI.
"""
