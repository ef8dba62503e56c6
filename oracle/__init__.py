"""CPU oracle for the LRI space-time RPA path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the method computes, written from
the paper's equations (arXiv:2407.19930, Sec. 2):

* ``green``      -- Eq. green_mat: G^occ / G^vir (R, tau) from KS eigen-data;
* ``chi0_definition`` -- Eqs. LRI + chi0_NAOs + chi0_ABFs written out with
  dense neighbourhood matrices (the plain definition of chi0_{mu nu}(R, tau));
* ``chi0_matrix`` -- the four-term matrix form of chi0_{mu nu}(R, tau) of Sec. 2
  (the equation combining Eqs. chi0_NAOs, chi0_ABFs and LRI), term by term in
  plain C with OpenMP over (point, atom pair); also the timed CPU baseline;
* ``chi0_sos``   -- an independent sum-over-states form in k space, used to
  pin the two routes above (exact in tau; Lorentzian in i omega);
* ``freq``       -- the tau -> i omega cosine transform and R -> q Fourier
  transform (Sec. 2, "RPA correlation energy");
* ``energy``     -- Tr[ln(1 - Pi) + Pi] through an LU factorisation of
  1 - chi0 V (the paper's route) and the E_c quadrature;
* ``grid``       -- minimax tau / omega grids and the cosine-transform weights;
* ``screen``     -- Green's-function block screening (Sec. 5's threshold; the
  block rule is a reading, stated in the module).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package.  The GPU library
never imports it, and it never imports the GPU library: the two share no
code.  Inputs come from ``paper_2407_19930_gb300.synthetic`` (a generator
module that holds none of the method's arithmetic) or are passed in.

Sign and unit conventions (the "real convention"): with the paper's
G(i tau) = +i G^vir(tau) for tau > 0 and G(-i tau) = -i G^occ(tau), the
product G(i tau) G(-i tau) is the real G^vir G^occ, so
chi0(tau) = -s G^vir(r, r', tau) G^occ(r', r, tau) with spin factor s = 2,
and chi0(i omega_k) = sum_j Gamma_kj chi0(tau_j) where the real matrix
Gamma_kj = gamma_jk cos(omega_k tau_j) absorbs the paper's -i factors and the
even extension in tau; chi0(i omega) is then real-symmetric in R space and
negative semidefinite in q space.
"""
