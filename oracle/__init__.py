"""Plain, slow FP64 CPU oracle for the SMC hot path of vSMC (arXiv 1306.5583).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

Every function follows the paper's definitions step by step, in float64
(or exact Python integers where the method is an integer procedure), with
no blocking, fusion or reordering beyond what the definition states.  It
shares no code with the CUDA path.

Modules
-------
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
          uniform / normal / exponential transforms (Sec. 3.4 "Third-party
          dependencies": one independent counter-based stream per particle).
weights   log-sum-exp normaliser, normalised weights, ESS (Sec. 2.1, ESS
          definition; Sec. 4.1.6 WeightSet), normalising-constant ratio
          (Sec. 2.2).
resample  fixed-point CDF and the four resamplers (Sec. 2.1, eq:resample and
          the replication counts R_i; Douc et al. 2005 schemes).
cv        the almost-constant-velocity tracking model and Algorithm 1
          (Sec. 5.1).
kalman    exact log-likelihood of the linear-Gaussian variant of that model
          (closed-form pin for the particle filter's evidence estimate).
gmm       Bayesian Gaussian mixture model, tempered targets (eq:geometry),
          Algorithm 2, the three-block random-walk Metropolis kernel, the
          standard (eq:smc-ds) and path-sampling (eq:path_est) estimators
          (Sec. 5.2).

Parity status of each function is stated in its module header.
"""
