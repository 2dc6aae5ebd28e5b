__kernel void gofs(__global int *data)
{
    data[get_local_id(0)] = (int)get_global_offset(0);
}
