"""GB300-native batched neutron-reflectivity forward model, log-likelihood and
exact gradient (arXiv 2509.06924) behind a C-ABI library."""
