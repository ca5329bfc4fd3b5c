"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package only *draws* inputs (numpy ``default_rng`` streams on the host, or a
seeded ``torch.Generator`` on a CUDA device for the full-size tensors).  It holds
none of the sketching arithmetic: no Khatri-Rao product, no MTTKRP, no QR of a
sketch, no core computation.  Both the FP64 oracle and the CUDA library receive
the arrays produced here as plain inputs.

Layout convention: a d-way tensor of dims (n_1, ..., n_d) is stored mode-1
fastest.  Host arrays are numpy arrays of shape (n_1, ..., n_d) in Fortran order;
device tensors are torch tensors of shape (n_d, ..., n_1), C-contiguous.  Both
describe the same bytes.
"""

from .tucker import (TuckerSpec, haar, tucker_factors, expand_tucker,
                     tucker_tensor, config_spec, to_torch_layout,
                     from_torch_layout)
from .hankel import (HankelSpec, markov_parameters, hankel_config_spec, symmetric_markov_parameters,
                     two_level_markov_parameters)
from .batch import batch_tucker_specs, batch_hankel_specs
from .cauchy import cauchy_tensor, cauchy_tensor_device

__all__ = [
    "TuckerSpec", "haar", "tucker_factors", "expand_tucker", "tucker_tensor",
    "config_spec", "to_torch_layout", "from_torch_layout", "HankelSpec",
    "markov_parameters", "hankel_config_spec", "symmetric_markov_parameters",
    "cauchy_tensor", "cauchy_tensor_device", "two_level_markov_parameters", "batch_tucker_specs", "batch_hankel_specs",
]
