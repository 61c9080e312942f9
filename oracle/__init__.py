"""FP64 CPU oracle for the reacting Navier-Stokes RHS and its SSP-RK3 step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, independent
restatement of the method against which the CUDA path is checked.  Only the
test suite, `__graft_entry__.smoke()` and the CPU-baseline / reference arm of
`bench.py` may import it; the product path never does.  It shares no code with
the CUDA library: the two meet only through the seeded inputs of
`paper_2202_02319_b300.synth`.

Everything is written with plain PyTorch CPU tensor operations in float64,
vectorised over cells, in the order the paper states each step:

  thermo      NASA polynomials, ideal-gas EOS, temperature from internal energy
  transport   Wilke mixture viscosity / conductivity, mixture-averaged diffusion
  chemistry   reversible Arrhenius mass-action rates, equilibrium constants
  laser       Gaussian space-time energy deposition
  fluxes      WENO3-Z with local Lax-Friedrichs splitting; 2nd-order central
              viscous, heat and species-diffusion fluxes
  rhs         cell state, source terms, flux divergence
  charwise    characteristic-wise flux splitting (the optional scheme variant)
  mapped      curvilinear grids: face area vectors, volumes, metrics, mapped fluxes
  nscbc       characteristic (NSCBC) inflow / outflow boundaries
  rk          SSP-RK3 (Shu-Osher form) and the time-step rule
  adjoint     discrete vector-Jacobian products by reverse-mode autodiff of the
              functions above

Where the paper is silent the oracle takes one stated reading; each module's
docstring lists the readings it implements.
"""
from . import thermo, transport, chemistry, laser, fluxes, charwise, mapped, nscbc, rhs, rk  # noqa: F401
from .mech import MechT, GridT, from_synth  # noqa: F401
