"""GB300-native lensless RF volumetric rendering (GeRaF hot path).

The compute path is the CUDA library ``libgeraf.so`` (C ABI in
``include/geraf.h``); this package only marshals torch tensors to it.
"""
from .geraf import (AnalyticField, Band, MLPField, make_grid, geraf_sample, geraf_fields,
                    geraf_fields_backward, geraf_blend, geraf_blend_backward, geraf_render,
                    geraf_render_backward, geraf_filter, geraf_filter_backward, geraf_poll_device_error,
                    geraf_check_bounded_wait,
                    geraf_render_noalloc, Proposal, geraf_proposal_density, geraf_sample_proposal, geraf_sample_cells,
                    geraf_sample_backward, geraf_chebyshev_order, geraf_chebyshev_work, geraf_masked_loss,
                    SAMPLE_UNIFORM, SAMPLE_STRATIFIED, PREC_FP32, PREC_BF16,
                    PHASOR_AUTO, PHASOR_RECURRENCE, PHASOR_CHEBYSHEV)
from ._lib import GerafError

__all__ = ["AnalyticField", "Band", "MLPField", "make_grid", "geraf_sample", "geraf_fields",
           "geraf_fields_backward", "geraf_blend", "geraf_blend_backward", "geraf_render",
           "geraf_render_backward", "geraf_filter", "geraf_filter_backward", "geraf_poll_device_error",
           "geraf_check_bounded_wait",
           "GerafError", "geraf_render_noalloc", "Proposal", "geraf_proposal_density", "geraf_sample_proposal",
           "geraf_sample_cells",
           "geraf_sample_backward", "geraf_chebyshev_order", "geraf_chebyshev_work", "geraf_masked_loss", "SAMPLE_UNIFORM", "SAMPLE_STRATIFIED", "PREC_FP32",
           "PREC_BF16", "PHASOR_AUTO", "PHASOR_RECURRENCE", "PHASOR_CHEBYSHEV"]
