"""FP64 CPU oracle of the nonlinear-damage ADER-DG step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, independent
restatement of the method (arXiv 2502.09714, Sec. 2 and Appendix A) in numpy
FP64.  Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the CUDA library never does, and it shares no code,
tables or helpers with the CUDA path (both only consume the seeded arrays of
the `synthetic` package).

Pins (see tests/test_oracle_*.py): quadrature exactness on monomials,
orthonormality/span of the basis, the stress as the strain gradient of an
energy, hand-derived damage rates of special strain states, the uniform-strain
closed form of damage growth, design-order convergence on the elastic plane
wave, energy decay, the brute-force monomial-basis re-derivation of one step,
invariance under relabelling/rotation/translation and monotone damage; for the
nonlinear shear law of the 1-D Riemann verification, its energy, plane-shear
reduction and secant moduli, and the exact Riemann solution's jump conditions,
invariants and linear limit; for the discrete adjoint (oracle/adjoint.py), its
pointwise derivatives, its step transpose and its misfit gradient against
central differences of the forward law, step and run.
"""
from .basis import eval_basis, mode_list, n_modes
from .quadrature import gauss_jacobi, gauss_legendre_01, tet_rule, tri_rule
from .rheology import (cdm_damage_rate, cdm_energy, cdm_stress, effective_lame, flux,
                       invariants, ivm_damage_rate, ivm_effective_lame, ivm_energy, ivm_stress,
                       jacobian_eff, nlshear_effective_lame, nlshear_energy, nlshear_stress)
from .riemann import ShearRiemann
from .solver import MeshError, Oracle, from_abi, stf_integral, to_abi

__all__ = [
    "eval_basis", "mode_list", "n_modes", "gauss_jacobi", "gauss_legendre_01", "tet_rule",
    "tri_rule", "cdm_damage_rate", "cdm_energy", "cdm_stress", "effective_lame", "flux",
    "invariants", "ivm_damage_rate", "ivm_effective_lame", "ivm_energy", "ivm_stress",
    "jacobian_eff", "nlshear_effective_lame", "nlshear_energy", "nlshear_stress", "ShearRiemann",
    "MeshError", "Oracle", "from_abi", "to_abi", "stf_integral",
]
