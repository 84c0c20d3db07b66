"""libhp: the NSHEDB homomorphic equality predicate (BFV, p = 65537) on one B300."""
